// ecmc_stripes.cu -- the striped decomposition that Sec. 3.4 tests beside
// the checkerboard (Fig. 3, "stripes"; interface and readings in
// ecmc_stripes.h).
//
// Per sweep: ks_begin (draws), ks_bin (stripe of every disk), one ks_phase
// launch per colour with one block per stripe of that colour, ks_end
// (deterministic sums).  A block builds its stripe's frame in global memory
// -- the members in ascending id, then every image across the axis of every
// other disk whose centre lies within sigma of the stripe's band, both by an
// ordered block-wide compaction over all disks -- and runs the stripe's n_m
// chains one after the other.  Per event every thread tests a strided share
// of the frame with the plain FP64 expressions of the variant (no
// contraction: the library is built with -fmad=false; sqrt and fmod are
// correctly rounded and exact), a block reduction takes the first hit by
// (distance, key), and thread 0 applies the event.  Only the coordinate
// along the axis changes, and a block writes only its own members', so the
// blocks of one colour never touch each other's data.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <climits>
#include <vector>

#include "ecmc.h"
#include "ecmc_stripes.h"
#include "ecmc_device.cuh"
#include "ecmc_internal.cuh"

namespace ecmcs {

using ecmc::U64x4;
using ecmc::below_n;
using ecmc::cell_1d;
using ecmc::philox;
using ecmc::unit_double;
using ecmc::wrap_half;

constexpr int kOk = 0, kCapacity = 1, kChainCap = 2;
constexpr int kThreads = 256, kWarps = kThreads / 32;
constexpr long long kMaxEvents = 1LL << 22;  // contacts of one chain
constexpr int kHistoryCap = 1 << 20;         // sweeps of pressure history kept

struct GeomS {
  int64_t N;
  double L, sigma, sig2, w, inv_w, ell;
  int S, n_m, reject;
  uint64_t seed, replica;
  int cap_obj;  // frame objects per stripe (packing bound of the band)
  int cap_mem;  // members per stripe (packing bound of the stripe itself)
  int list_mode;  // 0 start disks drawn with replacement, 1 shuffled list of distinct members
  // sorted-frame kernel: strips of width sw across the axis, nstrip of them
  double sw, inv_sw;
  int nstrip;
};

struct StateS {
  int64_t t;
  double shift;
  int first, axis;
};

struct StripeS {
  double sum_b;
  long long events, lifts, frozen, rejected;
  int chains, accepted, n_mem;
};

struct TotalsS {
  double sum_b, sum_disp, sum_b_w, sum_disp_w;
  long long sweeps, chains, events, lifts, frozen, rejected;
};

// position reduced into [0, L) (exact for values already inside)
__device__ __forceinline__ double wrap_along(double v, double L) {
  v = fmod(v, L);
  if (v < 0.0) v += L;
  if (v >= L) v -= L;
  return v;
}

__global__ void ks_begin(GeomS g, StateS* st) {
  if (threadIdx.x != 0) return;
  StateS s = *st;
  const U64x4 u = philox((uint64_t)s.t, ecmc::kPurposeSweep, 0, 0, g.seed, g.replica);
  s.shift = unit_double(u.v[0]) * g.w;
  s.first = (int)below_n(u.v[2], 2);
  s.axis = (int)(s.t & 1);
  *st = s;
}

__global__ void ks_bin(GeomS g, const StateS* __restrict__ st, const double* __restrict__ px,
                       const double* __restrict__ py, int* __restrict__ stripe_of) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.N) return;
  const StateS s = *st;
  const double v = s.axis ? px[i] : py[i];  // the coordinate across the axis
  stripe_of[i] = cell_1d(v, s.shift, g.L, g.inv_w, g.S);
}

// Block-ordered compaction step: every thread with `take` gets a slot
// base + (number of takers before it in thread order); returns the number
// of takers of the block.  Contains two barriers; call uniformly.
__device__ __forceinline__ int ordered_slot(bool take, int base, int* slot, int* wcnt) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned bal = __ballot_sync(0xffffffffu, take);
  if (lane == 0) wcnt[warp] = __popc(bal);
  __syncthreads();
  int before = 0, total = 0;
  for (int q = 0; q < kWarps; ++q) {
    before += q < warp ? wcnt[q] : 0;
    total += wcnt[q];
  }
  *slot = base + before + __popc(bal & ((1u << lane) - 1u));
  __syncthreads();  // wcnt is reused by the next call
  return total;
}

__global__ void __launch_bounds__(kThreads) ks_phase(
    GeomS g, const StateS* __restrict__ st, int ci, double* __restrict__ px,
    double* __restrict__ py, const int* __restrict__ stripe_of, double* __restrict__ fU,
    double* __restrict__ fV, long long* __restrict__ fkey, int* __restrict__ fid,
    double* __restrict__ fU0, StripeS* __restrict__ stats, int* __restrict__ recs, int* err) {
  __shared__ int wcnt[kWarps];
  __shared__ int sm_over, sm_m, sm_done;
  __shared__ double sm_d;
  __shared__ double red_s[kWarps];
  __shared__ long long red_k[kWarps];
  __shared__ int red_j[kWarps];

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const StateS s = *st;
  const int colour = ci == 0 ? s.first : 1 - s.first;
  const int a = blockIdx.x;        // active slot, 0 .. S/2 - 1
  const int k = colour + 2 * a;    // stripe index, < S
  double* along = s.axis ? py : px;
  const double* across = s.axis ? px : py;
  const double L = g.L, sigma = g.sigma, sig2 = g.sig2;
  const double origin = s.shift + (double)k * g.w;  // lower edge across
  const size_t fb = (size_t)a * (size_t)g.cap_obj;
  double* U = fU + fb;
  double* V = fV + fb;
  long long* key = fkey + fb;
  int* id = fid + fb;
  double* U0 = fU0 + fb;

  if (tid == 0) sm_over = 0;
  __syncthreads();

  // frame, part 1: the members in ascending id
  int n = 0;
  for (int64_t i0 = 0; i0 < g.N; i0 += kThreads) {
    const int64_t i = i0 + tid;
    const bool mem = i < g.N && stripe_of[i] == k;
    int slot;
    const int cnt = ordered_slot(mem, n, &slot, wcnt);
    if (mem) {
      if (slot < g.cap_obj) {
        U[slot] = along[i];
        V[slot] = wrap_half(across[i] - origin, L);
        key[slot] = (long long)i * 3 + 1;
        id[slot] = (int)i;
      } else {
        sm_over = 1;
      }
    }
    n += cnt;
  }
  const int n_mem = n;
  // frame, part 2: every image across (-L, 0, +L) of every other disk whose
  // centre lies within sigma of the band [0, w]
  for (int64_t i0 = 0; i0 < g.N; i0 += kThreads) {
    const int64_t i = i0 + tid;
    const bool other = i < g.N && stripe_of[i] != k;
    const double v0 = other ? wrap_half(across[i] - origin, L) : 0.0;
    for (int im = -1; im <= 1; ++im) {
      const double v = im == 0 ? v0 : (im > 0 ? v0 + L : v0 - L);
      const bool take = other && v > -sigma && v < g.w + sigma;
      int slot;
      const int cnt = ordered_slot(take, n, &slot, wcnt);
      if (take) {
        if (slot < g.cap_obj) {
          U[slot] = along[i];
          V[slot] = v;
          key[slot] = (long long)i * 3 + (im + 1);
          id[slot] = (int)i;
        } else {
          sm_over = 1;
        }
      }
      n += cnt;
    }
  }
  __syncthreads();
  const bool over = sm_over != 0;
  if (over && tid == 0) atomicCAS(err, kOk, kCapacity);

  // the chains
  double sum_b = 0.0;
  long long events = 0, lifts = 0, frozen = 0, rejected = 0;
  int chains = 0, accepted = 0;
  for (int c = 0; c < g.n_m; ++c) {
    int* rec = recs ? recs + ((size_t)k * g.n_m + c) * 4 : nullptr;
    if (over || n_mem == 0) {
      if (tid == 0 && rec) {
        rec[0] = -1;
        rec[1] = -1;
        rec[2] = 0;
        rec[3] = 0;
      }
      continue;  // uniform across the block
    }
    // thread 0 carries the chain's state; the others read m and d
    int m = 0;
    double d = 1.0, r = g.ell, chain_b = 0.0;
    long long nev = 0;
    if (tid == 0) {
      const U64x4 v = philox((uint64_t)s.t, ecmc::kPurposeChain, (uint64_t)k, (uint64_t)c,
                             g.seed, g.replica);
      m = (int)below_n(v.v[0], (uint64_t)n_mem);
      d = (v.v[1] >> 63) ? -1.0 : 1.0;
      if (rec) rec[0] = id[m];
      sm_m = m;
      sm_d = d;
      sm_done = 0;
    }
    if (g.reject)
      for (int q = tid; q < n_mem; q += kThreads) U0[q] = U[q];
    __syncthreads();
    for (long long iter = 0;; ++iter) {
      const int mm = sm_m;
      const double dd = sm_d;
      const double Um = U[mm], Vm = V[mm];
      double bs = INFINITY;
      long long bk = LLONG_MAX;
      int bj = -1;
      for (int j = tid; j < n; j += kThreads) {
        if (j == mm) continue;
        const double cc = V[j] - Vm;
        const double c2 = cc * cc;
        if (!(c2 < sig2)) continue;  // passes beside
        double b = dd * (U[j] - Um);
        if (b <= 0.0) b += L;        // ahead round the periodic stripe
        double sj = b - sqrt(sig2 - c2);
        if (sj < 0.0) sj = 0.0;
        const long long kj = key[j];
        if (sj < bs || (sj == bs && kj < bk)) {
          bs = sj;
          bk = kj;
          bj = j;
        }
      }
      for (int off = 16; off > 0; off >>= 1) {
        const double s2 = __shfl_xor_sync(0xffffffffu, bs, off);
        const long long k2 = __shfl_xor_sync(0xffffffffu, bk, off);
        const int j2 = __shfl_xor_sync(0xffffffffu, bj, off);
        if (s2 < bs || (s2 == bs && k2 < bk)) {
          bs = s2;
          bk = k2;
          bj = j2;
        }
      }
      if (lane == 0) {
        red_s[warp] = bs;
        red_k[warp] = bk;
        red_j[warp] = bj;
      }
      __syncthreads();
      if (tid == 0) {
        bs = red_s[0];
        bk = red_k[0];
        bj = red_j[0];
        for (int q = 1; q < kWarps; ++q)
          if (red_s[q] < bs || (red_s[q] == bs && red_k[q] < bk)) {
            bs = red_s[q];
            bk = red_k[q];
            bj = red_j[q];
          }
        int done = 0;
        if (iter >= kMaxEvents) {
          atomicCAS(err, kOk, kChainCap);
          done = 3;
        } else if (r <= bs) {  // budget used up: the chain ends
          U[m] = wrap_along(Um + d * r, L);
          sum_b += chain_b;
          done = 1;
        } else {
          nev++;
          events++;
          if (bj >= n_mem && g.reject) {  // frozen disk: rejected as a whole
            frozen++;
            rejected++;
            done = 2;
          } else {
            // separation along the axis at the contact, recomputed with the
            // expression of the search
            double b = d * (U[bj] - Um);
            if (b <= 0.0) b += L;
            U[m] = wrap_along(Um + d * bs, L);
            r = r - bs;
            chain_b += b - bs;
            if (bj < n_mem) {  // lift
              lifts++;
              m = bj;
            } else {           // frozen disk, reflecting rule: back along the axis
              frozen++;
              d = -d;
            }
          }
        }
        sm_m = m;
        sm_d = d;
        sm_done = done;
      }
      __syncthreads();
      if (sm_done) break;
    }
    const int done = sm_done;
    if (done == 2)
      for (int q = tid; q < n_mem; q += kThreads) U[q] = U0[q];
    if (tid == 0) {
      chains++;
      accepted += done == 2 ? 0 : 1;
      if (rec) {
        rec[1] = id[m];
        rec[2] = (int)nev;
        rec[3] = 0;
      }
    }
    __syncthreads();
  }

  // write back the members' coordinate along the axis
  if (!over)
    for (int q = tid; q < n_mem; q += kThreads) along[id[q]] = U[q];
  if (tid == 0) {
    StripeS o;
    o.sum_b = sum_b;
    o.events = events;
    o.lifts = lifts;
    o.frozen = frozen;
    o.rejected = rejected;
    o.chains = chains;
    o.accepted = accepted;
    o.n_mem = over ? 0 : n_mem;
    stats[k] = o;
  }
}

// ---- the sorted-frame kernel ----------------------------------------------
// One block per stripe builds the frame, then its first warp runs the chains
// with the frame in shared memory and no block barrier per event.
//
// Strips.  The frame is cut across the axis into strips of width sw = sigma/2
// (1 + 2^-30).  Two objects of one strip are less than sigma apart across,
// so a move along the axis can never carry one past the other: the cyclic
// order along the axis within a strip holds for the whole phase.  Each strip
// is sorted once, by (U, key), and kept as a rotated sorted array: logical
// index i sits at sstart[q] + (rot[q] + i) mod n_q, ascending in U.  A member
// that wraps round the periodic axis was the last (or first) of its strip,
// and becomes the first (or last): rot[q] moves by one.
//
// Search.  An object can be hit only if it lies within sigma across, that is
// in the strips q_m - 2 .. q_m + 2 (sw >= sigma/2), and ahead along d.  In each
// strip the lanes find the first object strictly ahead (a 6-ary search over
// the logical order), then test a window of six objects in the order the
// mover meets them, with the oracle's FP64 expressions.  The forward distance
// b only grows along that order, and s >= b - sigma, so a strip is finished
// once its last tested object has b - sigma above min(r, best s); otherwise
// the next six are tested.  The first hit is the minimum of (s, key) over
// the warp: the same object, distance and event as the full scan.
constexpr int kSortThreads = 512;
constexpr int kLanesPerStrip = 6;

__device__ __forceinline__ int strip_of_v(const GeomS& g, double v) {
  int q = (int)((v + g.sigma) * g.inv_sw);
  return q < 0 ? 0 : (q >= g.nstrip ? g.nstrip - 1 : q);
}

__host__ __device__ inline size_t sorted_smem_bytes(int cap_obj, int cap_mem, int nstrip) {
  return (sizeof(double) * 2 + sizeof(int) * 2) * (size_t)cap_obj + sizeof(int) * (size_t)cap_mem +
         sizeof(int) * (size_t)(3 * nstrip + 8) + ((size_t)cap_obj + 16);
}

__global__ void __launch_bounds__(kSortThreads) ks_phase_sorted(
    GeomS g, const StateS* __restrict__ st, int ci, double* __restrict__ px,
    double* __restrict__ py, const int* __restrict__ stripe_of, double* __restrict__ fU,
    double* __restrict__ fV, long long* __restrict__ fkey, int* __restrict__ fid,
    double* __restrict__ fU0, int* __restrict__ flist, StripeS* __restrict__ stats,
    int* __restrict__ recs, int* err) {
  extern __shared__ __align__(16) unsigned char ssm[];
  __shared__ int wcnt[kSortThreads / 32];
  __shared__ int sm_over, sm_n;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const unsigned FULL = 0xffffffffu;
  const StateS s = *st;
  const int colour = ci == 0 ? s.first : 1 - s.first;
  const int a = blockIdx.x;
  const int k = colour + 2 * a;
  double* along = s.axis ? py : px;
  const double* across = s.axis ? px : py;
  const double L = g.L, sigma = g.sigma, sig2 = g.sig2;
  const float g_sigf = (float)sigma;
  const double origin = s.shift + (double)k * g.w;
  const size_t fb = (size_t)a * (size_t)g.cap_obj;
  double* gU = fU + fb;
  double* gV = fV + fb;
  long long* gK = fkey + fb;
  int* gO = fid + fb;
  double* U0 = fU0 + (size_t)a * (size_t)g.cap_mem;
  int* plist = flist + (size_t)a * (size_t)g.cap_mem;

  // shared layout: U, V (double), key, orig (int) per object; the member map;
  // strip starts, rotations and their copy at a chain start
  double* U = (double*)ssm;
  double* V = U + g.cap_obj;
  int* key = (int*)(V + g.cap_obj);
  int* orig = key + g.cap_obj;
  int* mem_g = orig + g.cap_obj;
  int* sstart = mem_g + g.cap_mem;   // nstrip + 1
  int* rot = sstart + g.nstrip + 1;  // nstrip
  int* fill = rot + g.nstrip;        // nstrip (build), then rot at the chain start
  unsigned char* sq = (unsigned char*)(fill + g.nstrip);  // strip of every object

  if (tid == 0) sm_over = 0;
  for (int q = tid; q < g.nstrip; q += kSortThreads) fill[q] = 0;
  __syncthreads();

  // frame, part 1: the members in ascending id (unsorted, in global scratch)
  int n = 0;
  for (int64_t i0 = 0; i0 < g.N; i0 += kSortThreads) {
    const int64_t i = i0 + tid;
    const bool mem = i < g.N && stripe_of[i] == k;
    const unsigned bal = __ballot_sync(FULL, mem);
    if (lane == 0) wcnt[warp] = __popc(bal);
    __syncthreads();
    int before = 0, total = 0;
    for (int q = 0; q < kSortThreads / 32; ++q) {
      before += q < warp ? wcnt[q] : 0;
      total += wcnt[q];
    }
    const int slot = n + before + __popc(bal & ((1u << lane) - 1u));
    __syncthreads();
    if (mem) {
      if (slot < g.cap_mem) {
        gU[slot] = along[i];
        gV[slot] = wrap_half(across[i] - origin, L);
        gK[slot] = (long long)i * 3 + 1;
      } else {
        sm_over = 1;
      }
    }
    n += total;
  }
  const int n_mem = n;
  __syncthreads();
  // frame, part 2: images across (-L, 0, +L) of the other disks within sigma
  // of the band (any order: the strips are sorted by (U, key) below)
  if (tid == 0) sm_n = n_mem;
  __syncthreads();
  for (int64_t i = tid; i < g.N; i += kSortThreads) {
    if (stripe_of[i] == k) continue;
    const double v0 = wrap_half(across[i] - origin, L);
    for (int im = -1; im <= 1; ++im) {
      const double v = im == 0 ? v0 : (im > 0 ? v0 + L : v0 - L);
      if (!(v > -sigma && v < g.w + sigma)) continue;
      const int slot = atomicAdd(&sm_n, 1);
      if (slot < g.cap_obj) {
        gU[slot] = along[i];
        gV[slot] = v;
        gK[slot] = (long long)i * 3 + (im + 1);
      } else {
        sm_over = 1;
      }
    }
  }
  __syncthreads();
  const bool over = sm_over != 0;
  n = over ? 0 : sm_n;
  if (over && tid == 0) atomicCAS(err, kOk, kCapacity);

  // strips: counts, starts, then each object's rank within its strip by
  // (U, key); the sorted frame goes through global scratch into shared memory
  for (int o = tid; o < n; o += kSortThreads) atomicAdd(&fill[strip_of_v(g, gV[o])], 1);
  __syncthreads();
  if (tid == 0) {
    int acc = 0;
    for (int q = 0; q < g.nstrip; ++q) {
      sstart[q] = acc;
      acc += fill[q];
      fill[q] = 0;
      rot[q] = 0;
    }
    sstart[g.nstrip] = acc;
  }
  __syncthreads();
  for (int o = tid; o < n; o += kSortThreads) {
    const int q = strip_of_v(g, gV[o]);
    const int p = sstart[q] + atomicAdd(&fill[q], 1);
    U[p] = gU[o];
    V[p] = gV[o];
    key[p] = (int)gK[o];
    orig[p] = o;
  }
  __syncthreads();
  for (int q = 0; q < g.nstrip; ++q) {
    const int b0 = sstart[q], b1 = sstart[q + 1];
    for (int p = b0 + tid; p < b1; p += kSortThreads) {
      const double up = U[p];
      const int kp = key[p];
      int r = 0;
      for (int p2 = b0; p2 < b1; ++p2) r += (U[p2] < up || (U[p2] == up && key[p2] < kp));
      const int f = b0 + r;
      gU[f] = up;
      gV[f] = V[p];
      gK[f] = kp;
      gO[f] = orig[p];
    }
  }
  __syncthreads();
  for (int f = tid; f < n; f += kSortThreads) {
    U[f] = gU[f];
    V[f] = gV[f];
    key[f] = (int)gK[f];
    orig[f] = gO[f];
    sq[f] = (unsigned char)strip_of_v(g, gV[f]);
    if (gO[f] < n_mem) mem_g[gO[f]] = f;
  }
  __syncthreads();

  if (warp == 0) {
    double sum_b = 0.0;
    long long events = 0, lifts = 0, frozen = 0, rejected = 0;
    int chains = 0, accepted = 0;
    const int slot = lane / kLanesPerStrip, li = lane - slot * kLanesPerStrip;  // slot 5: idle
    const double INF = __longlong_as_double(0x7ff0000000000000ll);
    // shuffled list of distinct members (negative control), as the oracle
    // draws it: entry 0 as drawn, then Fisher-Yates on entries 1..
    if (g.list_mode == 1 && n_mem > 0 && !over && lane == 0) {
      const U64x4 v0 = philox((uint64_t)s.t, ecmc::kPurposeChain, (uint64_t)k, 0, g.seed,
                              g.replica);
      const int fst = (int)below_n(v0.v[0], (uint64_t)n_mem);
      int nr = 0;
      plist[nr++] = fst;
      for (int q = 0; q < n_mem; ++q)
        if (q != fst) plist[nr++] = q;
      U64x4 u;
      int cur = -1;
      for (int i = n_mem - 1; i >= 2; --i) {
        if ((i >> 2) != cur) {
          cur = i >> 2;
          u = philox((uint64_t)s.t, ecmc::kPurposeShuffle, (uint64_t)k, (uint64_t)cur, g.seed,
                     g.replica);
        }
        const int j = 1 + (int)below_n(u.v[i & 3], (uint64_t)i);
        const int tmp = plist[i];
        plist[i] = plist[j];
        plist[j] = tmp;
      }
    }
    __syncwarp();
    for (int c = 0; c < g.n_m; ++c) {
      int* rec = recs ? recs + ((size_t)k * g.n_m + c) * 4 : nullptr;
      if (over || n_mem == 0) {
        if (lane == 0 && rec) {
          rec[0] = -1;
          rec[1] = -1;
          rec[2] = 0;
          rec[3] = 0;
        }
        continue;
      }
      const U64x4 v = philox((uint64_t)s.t, ecmc::kPurposeChain, (uint64_t)k, (uint64_t)c,
                             g.seed, g.replica);
      const int q0 = g.list_mode == 1 ? plist[c % n_mem] : (int)below_n(v.v[0], (uint64_t)n_mem);
      int m = mem_g[q0];
      int dsg = (v.v[1] >> 63) ? -1 : 1;
      double d = dsg < 0 ? -1.0 : 1.0;
      double r = g.ell, chain_b = 0.0;
      long long nev = 0;
      if (lane == 0 && rec) rec[0] = key[m] / 3;
      if (g.reject) {
        for (int q = lane; q < n_mem; q += 32) U0[q] = U[mem_g[q]];
        for (int q = lane; q < g.nstrip; q += 32) fill[q] = rot[q];
      }
      __syncwarp();
      int done = 0;  // 1 budget used up, 2 rejected, 3 contact cap
      for (long long iter = 0;; ++iter) {
        const double Um = U[m], Vm = V[m];
        const long long kUm = ecmc::dkey(Um);
        const int qm = sq[m];
        // this lane's strip, its size and the first object strictly ahead
        const int q = qm - 2 + slot;
        const bool sv = slot < 5 && q >= 0 && q < g.nstrip;
        const int b0 = sv ? sstart[q] : 0;
        const int nq = sv ? sstart[q + 1] - b0 : 0;
        const int rq = sv ? rot[q] : 0;
        // first logical index with U > Um (d = +1) or U >= Um (d = -1), by a
        // 6-ary search over [lo, hi): the predicate is false ... false true ...
        // true (compared as order-preserving integers)
        int lo = 0, hi = nq;
        while (__any_sync(FULL, hi - lo > 0)) {
          const int len = hi - lo;
          const int step = (len + kLanesPerStrip) / (kLanesPerStrip + 1);  // >= 1
          const int probe = lo + (li + 1) * step - 1;
          bool pred = false;
          const bool act = sv && len > 0 && probe < hi;
          if (act) {
            int pi = rq + probe;
            pi -= pi >= nq ? nq : 0;
            const long long ku = ecmc::dkey(U[b0 + pi]);
            pred = dsg > 0 ? (ku > kUm) : (ku >= kUm);
          }
          const unsigned bt = __ballot_sync(FULL, act && pred);
          const unsigned bf = __ballot_sync(FULL, act && !pred);
          const unsigned gm = ((1u << kLanesPerStrip) - 1u) << (slot * kLanesPerStrip);
          const unsigned t_g = bt & gm, f_g = bf & gm;
          if (sv && len > 0) {
            // the true probes are a suffix of the probes: nf false probes put
            // the answer in [lo + nf step, first true probe] (or above the
            // last probe); the interval shrinks every round
            const int nf = __popc(f_g);
            const int nlo = lo + nf * step;
            const int nhi = t_g ? lo + (nf + 1) * step - 1 : hi;
            lo = nlo;
            hi = nhi < nlo ? nlo : nhi;
          }
        }
        // logical start of the scan: the first object ahead along d
        int c0 = 0;
        if (sv && nq > 0) c0 = dsg > 0 ? (lo < nq ? lo : 0) : (lo > 0 ? lo - 1 : nq - 1);
        auto object_at = [&](int off) {
          int lidx = dsg > 0 ? c0 + off : c0 - off;
          lidx += lidx >= nq ? -nq : (lidx < 0 ? nq : 0);
          int pi = rq + lidx;
          pi -= pi >= nq ? nq : 0;
          return b0 + pi;
        };
        // a strip is finished once its last tested object of window wi is too
        // far along to be hit before lim, or the window reached its end
        auto still_open = [&](int wi, double bl, double lim) {
          const int last = (nq - wi * kLanesPerStrip) < kLanesPerStrip
                               ? (nq - wi * kLanesPerStrip) - 1
                               : kLanesPerStrip - 1;
          const int src = slot * kLanesPerStrip + (last < 0 ? 0 : last);
          const double blast = __shfl_sync(FULL, bl, src < 32 ? src : 31);
          const bool end_of_strip = (wi + 1) * kLanesPerStrip >= nq;
          return sv && nq > 0 && !end_of_strip &&
                 !(blast - sigma * (1.0 + 1e-12) > lim + 4e-16 * L);
        };

        // window 0, screened: b, c^2 and x = sigma^2 - c^2 exactly as the
        // oracle forms them in FP64 (so the hit decision c^2 < sigma^2 is
        // exact; multiplying by d = +-1 is a sign flip, comparisons of these
        // values run on the integer pipes), s estimated in FP32:
        //   x truncated to FP32, then sqrtf: |root - sqrt(x)| <= 2^-23 sigma + 2^-63,
        //   b32 = b truncated to FP32: |b32 - b| <= 2^-23 b,
        //   b32 - root rounded in FP32: 2^-24 (b + sigma),
        // and the oracle's own rounding of b - sqrt(x): 2^-53 (b + sigma);
        // mg(b) = 2^-21 (b + sigma) + 2^-60 covers that with room to spare
        double bs = INF, bb = 0.0;
        int bk = INT_MAX, bj = -1;
        double bl0 = 0.0, b_c = 0.0, x_c = 0.0;
        float lo_c = __int_as_float(0x7f800000), hf = lo_c;
        int j_c = -1;
        bool cand = false;
        if (sv && li < nq) {
          const int j = object_at(li);
          double bj0 = ecmc::flip_if(U[j] - Um, dsg < 0);
          if (ecmc::dkey(bj0) <= 0) bj0 += L;  // ahead round the periodic stripe
          bl0 = bj0;
          if (j != m) {
            const double cc = V[j] - Vm;
            const double c2 = cc * cc;
            if (ecmc::lt_nn(c2, sig2)) {
              const double x = sig2 - c2;
              const float b32 = ecmc::to_float_trunc(bj0);
              const float se = b32 - sqrtf(ecmc::to_float_trunc(x));
              const float mgf = (b32 + g_sigf) * 0x1p-20f + 0x1p-60f;
              const float l = se - mgf, h = se + mgf;
              lo_c = l < 0.0f ? 0.0f : l;
              hf = h < 0.0f ? 0.0f : h;
              cand = true;
              b_c = bj0;
              x_c = x;
              j_c = j;
            }
          }
        }
        // the smallest upper bound over the warp (non-negative floats order
        // as their bit patterns)
        const float Hf = __uint_as_float(__reduce_min_sync(FULL, __float_as_uint(hf)));
        const float rf = ecmc::to_float_up_nn(r);
        const float limf = rf < Hf ? rf : Hf;
        const double lim0 = (double)limf;
        if (!__any_sync(FULL, still_open(0, bl0, lim0))) {
          // every strip is finished after window 0: the first hit is among
          // the candidates whose lower bound reaches min(r, Hf); evaluate
          // those with the oracle's expression
          const bool need = cand && lo_c <= limf;
          const unsigned nb = __ballot_sync(FULL, need);
          if (need) {
            bs = b_c - sqrt(x_c);
            if (bs < 0.0) bs = 0.0;
            bk = key[j_c];
            bj = j_c;
            bb = b_c;
          }
          if (__popc(nb) == 1) {
            const int w = __ffs(nb) - 1;
            bs = __shfl_sync(FULL, bs, w);
            bk = __shfl_sync(FULL, bk, w);
            bj = __shfl_sync(FULL, bj, w);
            bb = __shfl_sync(FULL, bb, w);
          } else if (nb != 0) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
              const double s2 = __shfl_xor_sync(FULL, bs, o);
              const int k2 = __shfl_xor_sync(FULL, bk, o);
              const int j2 = __shfl_xor_sync(FULL, bj, o);
              const double b2 = __shfl_xor_sync(FULL, bb, o);
              if (s2 < bs || (s2 == bs && k2 < bk)) {
                bs = s2;
                bk = k2;
                bj = j2;
                bb = b2;
              }
            }
          }
        } else {
          // some strip needs more than six objects (long free flights): the
          // exact search over windows of six, every candidate in FP64
          bool open = sv && nq > 0;
          for (int wi = 0; __any_sync(FULL, open); ++wi) {
            const int off = wi * kLanesPerStrip + li;
            const bool act = open && off < nq;
            double bl = 0.0;
            if (act) {
              const int j = object_at(off);
              double bj0 = d * (U[j] - Um);
              if (bj0 <= 0.0) bj0 += L;
              bl = bj0;
              if (j != m) {
                const double cc = V[j] - Vm;
                const double c2 = cc * cc;
                if (c2 < sig2) {
                  double sj = bj0 - sqrt(sig2 - c2);
                  if (sj < 0.0) sj = 0.0;
                  const int kj = key[j];
                  if (sj < bs || (sj == bs && kj < bk)) {
                    bs = sj;
                    bk = kj;
                    bj = j;
                    bb = bj0;
                  }
                }
              }
            }
            double ws = bs;
            int wk = bk;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
              const double s2 = __shfl_xor_sync(FULL, ws, o);
              const int k2 = __shfl_xor_sync(FULL, wk, o);
              if (s2 < ws || (s2 == ws && k2 < wk)) {
                ws = s2;
                wk = k2;
              }
            }
            const double lim = r < ws ? r : ws;
            const bool keep = still_open(wi, bl, lim);
            open = open && keep;
          }
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            const double s2 = __shfl_xor_sync(FULL, bs, o);
            const int k2 = __shfl_xor_sync(FULL, bk, o);
            const int j2 = __shfl_xor_sync(FULL, bj, o);
            const double b2 = __shfl_xor_sync(FULL, bb, o);
            if (s2 < bs || (s2 == bs && k2 < bk)) {
              bs = s2;
              bk = k2;
              bj = j2;
              bb = b2;
            }
          }
        }
        if (iter >= kMaxEvents) {
          if (lane == 0) atomicCAS(err, kOk, kChainCap);
          done = 3;
          break;
        }
        if (r <= bs) {  // budget used up: the chain ends
          const double x = Um + d * r;
          if (lane == 0) {
            U[m] = wrap_along(x, L);
            if (x >= L || x < 0.0) {
              const int nm_ = sstart[qm + 1] - sstart[qm];
              int rr = rot[qm] + (dsg > 0 ? nm_ - 1 : 1);
              rr -= rr >= nm_ ? nm_ : 0;
              rot[qm] = rr;
            }
          }
          sum_b += chain_b;
          done = 1;
          break;
        }
        nev++;
        events++;
        const bool is_member = orig[bj] < n_mem;
        if (!is_member && g.reject) {  // frozen disk: the chain is rejected
          frozen++;
          rejected++;
          done = 2;
          break;
        }
        // the move, with the wrap round the periodic axis: bs <= b <= L, so x
        // lies in (-L, 2L), where wrap_along is x - L (exact) or x + L
        const double x = Um + d * bs;
        const bool wrapped = (x >= L) || (x < 0.0);
        if (lane == 0) {
          U[m] = x >= L ? x - L : (x < 0.0 ? x + L : x);
          if (wrapped) {
            const int nm_ = sstart[qm + 1] - sstart[qm];
            int rr = rot[qm] + (dsg > 0 ? nm_ - 1 : 1);
            rr -= rr >= nm_ ? nm_ : 0;
            rot[qm] = rr;
          }
        }
        __syncwarp();
        r = r - bs;
        chain_b += bb - bs;
        if (is_member) {  // lift
          lifts++;
          m = bj;
        } else {          // frozen disk, reflecting rule: back along the axis
          frozen++;
          dsg = -dsg;
          d = -d;
        }
      }
      if (done == 2) {
        for (int q = lane; q < n_mem; q += 32) U[mem_g[q]] = U0[q];
        for (int q = lane; q < g.nstrip; q += 32) rot[q] = fill[q];
      }
      __syncwarp();
      chains++;
      accepted += done == 2 ? 0 : 1;
      if (lane == 0 && rec) {
        rec[1] = key[m] / 3;
        rec[2] = (int)nev;
        rec[3] = 0;
      }
    }
    if (lane == 0) {
      StripeS o;
      o.sum_b = sum_b;
      o.events = events;
      o.lifts = lifts;
      o.frozen = frozen;
      o.rejected = rejected;
      o.chains = chains;
      o.accepted = accepted;
      o.n_mem = over ? 0 : n_mem;
      stats[k] = o;
    }
  }
  __syncthreads();
  // write back the members' coordinate along the axis
  if (!over)
    for (int q = tid; q < n_mem; q += kSortThreads) {
      const int f = mem_g[q];
      along[key[f] / 3] = U[f];
    }
}

__global__ void ks_end(GeomS g, StateS* st, const StripeS* __restrict__ stats, TotalsS* tot,
                       double* history, int64_t* hist_len) {
  if (threadIdx.x != 0) return;
  TotalsS T = *tot;
  double bw = 0.0, dw = 0.0;
  for (int k = 0; k < g.S; ++k) {
    const StripeS o = stats[k];
    T.sum_b += o.sum_b;
    T.sum_disp += (double)o.accepted * g.ell;
    bw += (double)o.n_mem * o.sum_b;
    dw += (double)o.n_mem * ((double)o.accepted * g.ell);
    T.chains += o.chains;
    T.events += o.events;
    T.lifts += o.lifts;
    T.frozen += o.frozen;
    T.rejected += o.rejected;
  }
  T.sum_b_w += bw;
  T.sum_disp_w += dw;
  T.sweeps++;
  *tot = T;
  const int64_t h = *hist_len;
  if (h < kHistoryCap) {
    history[2 * h] = bw;
    history[2 * h + 1] = dw;
    *hist_len = h + 1;
  }
  st->t += 1;
}

__global__ void ks_split(const double* __restrict__ xy, int64_t N, double L,
                         double* __restrict__ px, double* __restrict__ py) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  px[i] = wrap_along(xy[2 * i], L);
  py[i] = wrap_along(xy[2 * i + 1], L);
}

__global__ void ks_join(const double* __restrict__ px, const double* __restrict__ py, int64_t N,
                        double* __restrict__ xy) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  xy[2 * i] = px[i];
  xy[2 * i + 1] = py[i];
}

}  // namespace ecmcs

// ---- host side ----------------------------------------------------------------

using namespace ecmcs;

struct ecmc_stripes_ctx {
  GeomS g;
  cudaStream_t stream = nullptr, own = nullptr;
  double *px = nullptr, *py = nullptr, *xy_tmp = nullptr;
  int *stripe_of = nullptr, *err = nullptr, *recs = nullptr;
  double *fU = nullptr, *fV = nullptr, *fU0 = nullptr;
  long long* fkey = nullptr;
  int* fid = nullptr;
  StripeS* stats = nullptr;
  StateS* st = nullptr;
  TotalsS* tot = nullptr;
  double* history = nullptr;
  int64_t* hist_len = nullptr;
  int* flist = nullptr;  // shuffled start lists, cap_mem per active stripe
  int64_t t_host = 0;
  bool valid = false;
  int kernel_param = 1;   // 1 sorted frames when they fit, 0 block-wide scan
  size_t sorted_smem = 0;
  bool sorted_ok = false; // the sorted frame fits in shared memory
};

namespace {

int fails(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  return ecmc::report_error(code, buf);
}

#define CKS(call)                                                                         \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return fails(e_ == cudaErrorMemoryAllocation ? ECMC_ERR_OOM : ECMC_ERR_CUDA,        \
                   "%s failed: %s", #call, cudaGetErrorString(e_));                       \
  } while (0)

// Frame objects of one stripe: images of pairwise non-overlapping disks
// (centre distance >= sigma) with centres in the band (-sigma, w + sigma)
// across, periodic with period L along; the disks of radius sigma / 2
// around them are disjoint and lie in a band of width w + 3 sigma and area
// (w + 3 sigma) L, so there are at most 4 (w + 3 sigma) L / (pi sigma^2).
int64_t frame_bound(double w, double L, double sigma) {
  const double b = 4.0 * (w + 3.0 * sigma) * L / (M_PI * sigma * sigma);
  return (int64_t)std::floor(b) + 2;
}

// Members of one stripe: centres in a band of width w, disks of radius
// sigma / 2 in a band of width w + sigma: at most 4 (w + sigma) L / (pi sigma^2).
int64_t member_bound(double w, double L, double sigma) {
  const double b = 4.0 * (w + sigma) * L / (M_PI * sigma * sigma);
  return (int64_t)std::floor(b) + 2;
}

bool use_sorted(const ecmc_stripes_ctx* h) { return h->kernel_param == 1 && h->sorted_ok; }

int checks(ecmc_stripes_ctx* h) {
  int e = 0;
  CKS(cudaMemcpyAsync(&e, h->err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CKS(cudaStreamSynchronize(h->stream));
  if (e == kCapacity) {
    h->valid = false;
    return fails(ECMC_ERR_CAPACITY, "a stripe's frame exceeded its packing bound");
  }
  if (e == kChainCap) {
    h->valid = false;
    return fails(ECMC_ERR_CHAIN_CAP, "a chain reached the per-chain contact cap");
  }
  return ECMC_OK;
}

int enqueue_sweep(ecmc_stripes_ctx* h, bool records) {
  const GeomS& g = h->g;
  const unsigned nb = (unsigned)((g.N + 255) / 256);
  ks_begin<<<1, 32, 0, h->stream>>>(g, h->st);
  ks_bin<<<nb, 256, 0, h->stream>>>(g, h->st, h->px, h->py, h->stripe_of);
  if (g.list_mode == 1 && !use_sorted(h))
    return fails(ECMC_ERR_UNSUPPORTED,
                 "shuffled start lists need the sorted-frame kernel, whose frame does not fit");
  for (int ci = 0; ci < 2; ++ci) {
    if (use_sorted(h))
      ks_phase_sorted<<<(unsigned)(g.S / 2), kSortThreads, h->sorted_smem, h->stream>>>(
          g, h->st, ci, h->px, h->py, h->stripe_of, h->fU, h->fV, h->fkey, h->fid, h->fU0,
          h->flist, h->stats, records ? h->recs : nullptr, h->err);
    else
      ks_phase<<<(unsigned)(g.S / 2), kThreads, 0, h->stream>>>(
          g, h->st, ci, h->px, h->py, h->stripe_of, h->fU, h->fV, h->fkey, h->fid, h->fU0,
          h->stats, records ? h->recs : nullptr, h->err);
  }
  ks_end<<<1, 32, 0, h->stream>>>(g, h->st, h->stats, h->tot, h->history, h->hist_len);
  CKS(cudaGetLastError());
  return ECMC_OK;
}

int load_dev(ecmc_stripes_ctx* h, const double* xy_dev, int64_t t0) {
  const GeomS& g = h->g;
  ks_split<<<(unsigned)((g.N + 255) / 256), 256, 0, h->stream>>>(xy_dev, g.N, g.L, h->px,
                                                                 h->py);
  CKS(cudaGetLastError());
  StateS s;
  std::memset(&s, 0, sizeof(s));
  s.t = t0;
  CKS(cudaMemcpyAsync(h->st, &s, sizeof(s), cudaMemcpyHostToDevice, h->stream));
  CKS(cudaMemsetAsync(h->tot, 0, sizeof(TotalsS), h->stream));
  CKS(cudaMemsetAsync(h->hist_len, 0, sizeof(int64_t), h->stream));
  CKS(cudaMemsetAsync(h->err, 0, sizeof(int), h->stream));
  CKS(cudaStreamSynchronize(h->stream));
  h->t_host = t0;
  h->valid = true;
  return ECMC_OK;
}

void frees(ecmc_stripes_ctx* h) {
  cudaFree(h->px);
  cudaFree(h->py);
  cudaFree(h->xy_tmp);
  cudaFree(h->stripe_of);
  cudaFree(h->err);
  cudaFree(h->recs);
  cudaFree(h->fU);
  cudaFree(h->fV);
  cudaFree(h->fU0);
  cudaFree(h->fkey);
  cudaFree(h->fid);
  cudaFree(h->stats);
  cudaFree(h->st);
  cudaFree(h->tot);
  cudaFree(h->history);
  cudaFree(h->hist_len);
  cudaFree(h->flist);
  if (h->own) cudaStreamDestroy(h->own);
}

}  // namespace

extern "C" {

int ecmc_stripes_create(ecmc_stripes_t* out, int64_t N, double L, double sigma, int stripes,
                        double ell, uint64_t seed) {
  if (!out) return fails(ECMC_ERR_ARG, "NULL output handle");
  *out = nullptr;
  // a frame holds at most 3 N objects, counted in int
  if (N < 1 || N >= (int64_t(1) << 29)) return fails(ECMC_ERR_ARG, "N out of range");
  int64_t k = (int64_t)std::llround(std::sqrt((double)N));
  while (k * k > N) --k;
  while ((k + 1) * (k + 1) <= N) ++k;
  if (k * k != N) return fails(ECMC_ERR_ARG, "N must be a perfect square (lattice start)");
  if (!(L > 0.0) || !(sigma > 0.0) || !std::isfinite(L) || !std::isfinite(sigma))
    return fails(ECMC_ERR_ARG, "L and sigma must be positive");
  if (!(sigma >= std::ldexp(1.0, -40) && sigma <= std::ldexp(1.0, 40) &&
        L < std::ldexp(sigma, 40)))
    return fails(ECMC_ERR_ARG, "sigma must lie in [2^-40, 2^40] and L below 2^40 sigma");
  if (stripes < 2 || (stripes & 1) || stripes > (1 << 20))
    return fails(ECMC_ERR_ARG, "stripes must be even, >= 2 and <= 2^20");
  if (!(L / (double)stripes > sigma)) return fails(ECMC_ERR_ARG, "stripe width must exceed sigma");
  if (!(L / (double)k > sigma)) return fails(ECMC_ERR_ARG, "square lattice would overlap");
  if (!(ell >= 0.0) || !std::isfinite(ell)) return fails(ECMC_ERR_ARG, "ell must be >= 0");
  const double w = L / (double)stripes;
  const int64_t cap = frame_bound(w, L, sigma);
  if (cap >= (int64_t(1) << 31) || (double)cap * (stripes / 2) > 4.0e9)
    return fails(ECMC_ERR_ARG, "stripe frames too large");
  ecmc_stripes_ctx* h = new ecmc_stripes_ctx();
  GeomS& g = h->g;
  std::memset(&g, 0, sizeof(g));
  g.N = N;
  g.L = L;
  g.sigma = sigma;
  g.sig2 = sigma * sigma;
  g.w = w;
  g.inv_w = 1.0 / w;
  g.ell = ell;
  g.S = stripes;
  g.n_m = 1;
  g.reject = 1;
  g.seed = seed;
  g.replica = 0;
  g.cap_obj = (int)cap;
  const int64_t capm = member_bound(w, L, sigma);
  g.cap_mem = (int)(capm < cap ? capm : cap);
  g.list_mode = 0;
  g.sw = 0.5 * sigma * (1.0 + std::ldexp(1.0, -30));
  g.inv_sw = 1.0 / g.sw;
  g.nstrip = (int)std::ceil((w + 2.0 * sigma) / g.sw) + 2;
  h->sorted_smem = sorted_smem_bytes(g.cap_obj, g.cap_mem, g.nstrip);
  {
    int dev = 0, optin = 0;
    cudaFuncAttributes fa;
    h->sorted_ok = cudaGetDevice(&dev) == cudaSuccess &&
                   cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin,
                                          dev) == cudaSuccess &&
                   cudaFuncGetAttributes(&fa, ks_phase_sorted) == cudaSuccess &&
                   h->sorted_smem + fa.sharedSizeBytes <= (size_t)optin &&
                   cudaFuncSetAttribute(ks_phase_sorted,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)h->sorted_smem) == cudaSuccess;
    cudaGetLastError();
  }
  if (cudaStreamCreateWithFlags(&h->own, cudaStreamNonBlocking) != cudaSuccess) {
    delete h;
    return fails(ECMC_ERR_CUDA, "stream creation failed");
  }
  h->stream = h->own;
  const size_t nn = (size_t)N, nf = (size_t)(stripes / 2) * (size_t)cap;
  if (cudaMalloc(&h->px, sizeof(double) * nn) != cudaSuccess ||
      cudaMalloc(&h->py, sizeof(double) * nn) != cudaSuccess ||
      cudaMalloc(&h->xy_tmp, sizeof(double) * 2 * nn) != cudaSuccess ||
      cudaMalloc(&h->stripe_of, sizeof(int) * nn) != cudaSuccess ||
      cudaMalloc(&h->err, sizeof(int)) != cudaSuccess ||
      cudaMalloc(&h->fU, sizeof(double) * nf) != cudaSuccess ||
      cudaMalloc(&h->fV, sizeof(double) * nf) != cudaSuccess ||
      cudaMalloc(&h->fU0, sizeof(double) * nf) != cudaSuccess ||
      cudaMalloc(&h->fkey, sizeof(long long) * nf) != cudaSuccess ||
      cudaMalloc(&h->fid, sizeof(int) * nf) != cudaSuccess ||
      cudaMalloc(&h->stats, sizeof(StripeS) * (size_t)stripes) != cudaSuccess ||
      cudaMalloc(&h->st, sizeof(StateS)) != cudaSuccess ||
      cudaMalloc(&h->tot, sizeof(TotalsS)) != cudaSuccess ||
      cudaMalloc(&h->history, sizeof(double) * 2 * kHistoryCap) != cudaSuccess ||
      cudaMalloc(&h->hist_len, sizeof(int64_t)) != cudaSuccess ||
      cudaMalloc(&h->flist, sizeof(int) * (size_t)(stripes / 2) * (size_t)g.cap_mem) !=
          cudaSuccess) {
    cudaGetLastError();
    frees(h);
    delete h;
    return fails(ECMC_ERR_OOM, "device allocation failed");
  }
  // the square lattice start: disk iy k + ix at ((ix + 1/2) a, (iy + 1/2) a)
  std::vector<double> xy(2 * nn);
  const double a = L / (double)k;
  for (int64_t i = 0; i < N; ++i) {
    xy[2 * i] = ((double)(i % k) + 0.5) * a;
    xy[2 * i + 1] = ((double)(i / k) + 0.5) * a;
  }
  const int rc = ecmc_stripes_set_positions(h, xy.data(), 0, 0);
  if (rc) {
    frees(h);
    delete h;
    return rc;
  }
  *out = h;
  return ECMC_OK;
}

int ecmc_stripes_destroy(ecmc_stripes_t h) {
  if (!h) return ECMC_OK;
  if (h->stream) cudaStreamSynchronize(h->stream);
  frees(h);
  delete h;
  return ECMC_OK;
}

int ecmc_stripes_set_param(ecmc_stripes_t h, int key, double v) {
  if (!h) return fails(ECMC_ERR_ARG, "NULL handle");
  switch (key) {
    case ECMC_STRIPES_PARAM_N_CHAINS: {
      const int n = (int)v;
      if ((double)n != v || n < 1 || n > (1 << 20)) return fails(ECMC_ERR_ARG, "n_m");
      if (n != h->g.n_m) {
        CKS(cudaStreamSynchronize(h->stream));
        h->g.n_m = n;
        cudaFree(h->recs);
        h->recs = nullptr;
      }
      return ECMC_OK;
    }
    case ECMC_STRIPES_PARAM_REPLICA:
      if (!(v >= 0.0) || v != std::floor(v) || v > 9.0e15) return fails(ECMC_ERR_ARG, "replica");
      h->g.replica = (uint64_t)v;
      return ECMC_OK;
    case ECMC_STRIPES_PARAM_BOUNDARY:
      if (v != (double)ECMC_BOUNDARY_REFLECT && v != (double)ECMC_BOUNDARY_REJECT)
        return fails(ECMC_ERR_ARG, "boundary must be ECMC_BOUNDARY_REFLECT or _REJECT");
      h->g.reject = v == (double)ECMC_BOUNDARY_REJECT ? 1 : 0;
      return ECMC_OK;
    case ECMC_STRIPES_PARAM_LIST_MODE:
      if (v != (double)ECMC_LIST_WITH_REPL && v != (double)ECMC_LIST_WITHOUT_REPL)
        return fails(ECMC_ERR_ARG, "list mode must be ECMC_LIST_WITH_REPL or _WITHOUT_REPL");
      h->g.list_mode = v == (double)ECMC_LIST_WITHOUT_REPL ? 1 : 0;
      return ECMC_OK;
    case ECMC_STRIPES_PARAM_KERNEL:
      if (v != 0.0 && v != 1.0) return fails(ECMC_ERR_ARG, "kernel must be 0 or 1");
      h->kernel_param = (int)v;
      return ECMC_OK;
    default:
      return fails(ECMC_ERR_ARG, "unknown parameter %d", key);
  }
}

int ecmc_stripes_get_param(ecmc_stripes_t h, int key, double* v) {
  if (!h || !v) return fails(ECMC_ERR_ARG, "NULL argument");
  switch (key) {
    case ECMC_STRIPES_PARAM_N_CHAINS: *v = h->g.n_m; return ECMC_OK;
    case ECMC_STRIPES_PARAM_REPLICA: *v = (double)h->g.replica; return ECMC_OK;
    case ECMC_STRIPES_PARAM_BOUNDARY:
      *v = h->g.reject ? ECMC_BOUNDARY_REJECT : ECMC_BOUNDARY_REFLECT;
      return ECMC_OK;
    case ECMC_STRIPES_PARAM_LIST_MODE: *v = h->g.list_mode; return ECMC_OK;
    case ECMC_STRIPES_PARAM_KERNEL: *v = use_sorted(h) ? 1.0 : 0.0; return ECMC_OK;
    default: return fails(ECMC_ERR_ARG, "unknown parameter %d", key);
  }
}

int ecmc_stripes_set_stream(ecmc_stripes_t h, void* stream) {
  if (!h) return fails(ECMC_ERR_ARG, "NULL handle");
  CKS(cudaStreamSynchronize(h->stream));
  h->stream = stream ? (cudaStream_t)stream : h->own;
  return ECMC_OK;
}

int ecmc_stripes_set_positions(ecmc_stripes_t h, const double* xy, int on_device, int64_t t0) {
  if (!h || !xy) return fails(ECMC_ERR_ARG, "NULL argument");
  if (t0 < 0) return fails(ECMC_ERR_ARG, "t0 must be >= 0");
  const double* src = xy;
  if (!on_device) {
    CKS(cudaMemcpyAsync(h->xy_tmp, xy, sizeof(double) * 2 * (size_t)h->g.N,
                        cudaMemcpyHostToDevice, h->stream));
    src = h->xy_tmp;
  }
  return load_dev(h, src, t0);
}

int ecmc_stripes_positions(ecmc_stripes_t h, double* xy, int on_device) {
  if (!h || !xy) return fails(ECMC_ERR_ARG, "NULL argument");
  if (!h->valid) return fails(ECMC_ERR_STATE, "state invalid after an earlier error");
  const GeomS& g = h->g;
  double* dst = on_device ? xy : h->xy_tmp;
  ks_join<<<(unsigned)((g.N + 255) / 256), 256, 0, h->stream>>>(h->px, h->py, g.N, dst);
  CKS(cudaGetLastError());
  if (!on_device)
    CKS(cudaMemcpyAsync(xy, h->xy_tmp, sizeof(double) * 2 * (size_t)g.N, cudaMemcpyDeviceToHost,
                        h->stream));
  return checks(h);
}

int ecmc_stripes_sweep(ecmc_stripes_t h, int64_t n) {
  if (!h) return fails(ECMC_ERR_ARG, "NULL handle");
  if (n < 0) return fails(ECMC_ERR_ARG, "negative sweep count");
  if (!h->valid) return fails(ECMC_ERR_STATE, "state invalid after an earlier error");
  if (n > 0 && !h->recs)
    CKS(cudaMalloc(&h->recs, sizeof(int) * 4 * (size_t)h->g.S * (size_t)h->g.n_m));
  for (int64_t s = 0; s < n; ++s) {
    const int rc = enqueue_sweep(h, s == n - 1);
    if (rc) return rc;
  }
  h->t_host += n;
  return ECMC_OK;
}

int ecmc_stripes_synchronize(ecmc_stripes_t h) {
  if (!h) return fails(ECMC_ERR_ARG, "NULL handle");
  return checks(h);
}

int ecmc_stripes_sweep_index(ecmc_stripes_t h, int64_t* t) {
  if (!h || !t) return fails(ECMC_ERR_ARG, "NULL argument");
  *t = h->t_host;
  return ECMC_OK;
}

int ecmc_stripes_counters(ecmc_stripes_t h, ecmc_counters_t* out) {
  if (!h || !out) return fails(ECMC_ERR_ARG, "NULL argument");
  TotalsS t;
  CKS(cudaMemcpyAsync(&t, h->tot, sizeof(t), cudaMemcpyDeviceToHost, h->stream));
  const int rc = checks(h);
  if (rc) return rc;
  std::memset(out, 0, sizeof(*out));
  out->sweeps = t.sweeps;
  out->chains = t.chains;
  out->events = t.events;
  out->lifts = t.lifts;
  out->frozen_hits = t.frozen;
  out->wall_hits = 0;
  out->sum_b = t.sum_b;
  out->sum_disp = t.sum_disp;
  out->rejected_chains = t.rejected;
  return ECMC_OK;
}

int ecmc_stripes_pressure(ecmc_stripes_t h, double* betaP, double* se) {
  if (!h || !betaP) return fails(ECMC_ERR_ARG, "NULL argument");
  TotalsS t;
  int64_t n = 0;
  CKS(cudaMemcpyAsync(&t, h->tot, sizeof(t), cudaMemcpyDeviceToHost, h->stream));
  CKS(cudaMemcpyAsync(&n, h->hist_len, sizeof(n), cudaMemcpyDeviceToHost, h->stream));
  const int rc = checks(h);
  if (rc) return rc;
  if (n < 1 || !(t.sum_disp_w > 0.0))
    return fails(ECMC_ERR_STATE, "no accepted chain since the last reset");
  const GeomS& g = h->g;
  const double rho_s2 = (double)g.N / (g.L * g.L) * g.sig2;
  *betaP = rho_s2 * (1.0 + t.sum_b_w / t.sum_disp_w);
  if (se) {
    *se = 0.0;
    const int64_t m = n < kHistoryCap ? n : kHistoryCap;
    const int64_t nb = m >= 20 ? 20 : m;
    if (nb >= 2) {
      std::vector<double> hist(2 * (size_t)m);
      CKS(cudaMemcpyAsync(hist.data(), h->history, sizeof(double) * 2 * (size_t)m,
                          cudaMemcpyDeviceToHost, h->stream));
      CKS(cudaStreamSynchronize(h->stream));
      std::vector<double> vals;
      for (int64_t b = 0; b < nb; ++b) {
        const int64_t lo = b * m / nb, hi = (b + 1) * m / nb;
        double sb = 0.0, sd = 0.0;
        for (int64_t i = lo; i < hi; ++i) {
          sb += hist[2 * i];
          sd += hist[2 * i + 1];
        }
        if (sd > 0.0) vals.push_back(rho_s2 * (1.0 + sb / sd));
      }
      const size_t nv = vals.size();
      if (nv >= 2) {
        double mean = 0.0;
        for (double v : vals) mean += v;
        mean /= (double)nv;
        double var = 0.0;
        for (double v : vals) var += (v - mean) * (v - mean);
        *se = std::sqrt(var / (double)(nv - 1) / (double)nv);
      }
    }
  }
  return ECMC_OK;
}

int ecmc_stripes_reset_stats(ecmc_stripes_t h) {
  if (!h) return fails(ECMC_ERR_ARG, "NULL handle");
  CKS(cudaMemsetAsync(h->tot, 0, sizeof(TotalsS), h->stream));
  CKS(cudaMemsetAsync(h->hist_len, 0, sizeof(int64_t), h->stream));
  return ECMC_OK;
}

int ecmc_stripes_last_stripes(ecmc_stripes_t h, int32_t* stripe_of_id) {
  if (!h || !stripe_of_id) return fails(ECMC_ERR_ARG, "NULL argument");
  CKS(cudaMemcpyAsync(stripe_of_id, h->stripe_of, sizeof(int32_t) * (size_t)h->g.N,
                      cudaMemcpyDeviceToHost, h->stream));
  return checks(h);
}

int ecmc_stripes_chain_records(ecmc_stripes_t h, int32_t* out) {
  if (!h || !out) return fails(ECMC_ERR_ARG, "NULL argument");
  if (!h->recs) return fails(ECMC_ERR_STATE, "no sweep has run");
  CKS(cudaMemcpyAsync(out, h->recs, sizeof(int32_t) * 4 * (size_t)h->g.S * (size_t)h->g.n_m,
                      cudaMemcpyDeviceToHost, h->stream));
  return checks(h);
}

}  // extern "C"
