// ecmc3.cu -- the parallel event-chain sweep for hard spheres in three
// dimensions (the generalisation of Sec. 3.4 to cubic cells in 2x2x2 blocks;
// interface and readings in ecmc3.h).
//
// Per sweep: k3_begin (draws), k3_bin (bucket every sphere by cell), the
// eight colour phases -- one persistent k3_sweep launch by default, or eight
// k3_phase launches -- and k3_end (deterministic sums).  Either way one warp
// processes one active cell (cell3): it sorts the cell's members by id,
// gathers the members and every periodic image of the 26 neighbour cells'
// spheres within sigma of the cell into a shared-memory frame (FP64
// coordinates and their FP32 roundings), bins the frame across the sweep's
// axis, and runs the cell's n_m chains.  Each event takes the three rows of
// bins around the mover, screens their spheres in FP32 with a rigorous
// margin (a sphere behind the mover or with perpendicular offset >= sigma
// cannot be hit), tests the survivors in FP64 with the oracle's expressions
// (no contraction: the library is built with -fmad=false) in one warp-wide
// pass, and a shuffle reduction picks the first hit by (distance, key).  As
// in the two-dimensional loop, comparisons of FP64 values and the square
// root run on the integer pipes (bit-pattern orders, the correctly rounded
// sqrt_rn): the same results as the FP64 instructions, with the FP64 pipe
// left the arithmetic.  Positions live in sphere-id order; a cell reads its
// frozen neighbours' positions, which no warp writes while it runs (later
// colours wait for it, earlier ones have finished).
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <climits>
#include <vector>

#include "ecmc.h"
#include "ecmc3.h"
#include "ecmc_device.cuh"
#include "ecmc_internal.cuh"

namespace ecmc3 {

using ecmc::U64x4;
using ecmc::below_n;
using ecmc::cell_1d;
using ecmc::clamp0;
using ecmc::dbits;
using ecmc::dlt;
using ecmc::flip_if;
using ecmc::le_nn;
using ecmc::lt_nn;
using ecmc::philox;
using ecmc::plus_zero;
using ecmc::sqrt_rn;
using ecmc::to_float_trunc;
using ecmc::unit_double;
using ecmc::wrap_box0;
using ecmc::wrap_half;
using ecmc::wrap_half_i;

constexpr int kOk = 0, kCapacity = 1, kChainCap = 2, kWaitTimeout = 4;
constexpr int kWarpsMax = 4;
constexpr int kHistoryCap = 1 << 20;  // sweeps of pressure history kept

struct Geom3 {
  int64_t N;
  double L, sigma, sig2, w, inv_w, ell;
  int cells, ncell, nact, n_m;
  uint64_t seed, replica;
  int cap_mem, cap_obj;  // bucket slots per cell; frame objects per cell
  int warp_bytes;        // shared memory of one warp's frame
  // FP32 screen: frame coordinates lie in (-sigma, w + sigma) and are
  // truncated to FP32 (integer pipes) with error < 2^-23 M (M >= w + sigma),
  // so FP32 differences (two truncations and one FP32 rounding of at most
  // 2^-24 2M) are within d = 8 2^-24 M of the FP64 ones; a hit (b > 0,
  // c^2 < sigma^2) then has b32 > -d and c2_32 < sigma^2 + 4 d sigma +
  // 2 d^2 + FP32 rounding; the thresholds below are twice those bounds
  float scr_b;           // pass iff b32 > -scr_b
  float scr_c2;          // pass iff c2_32 < scr_c2
  // L >= 2 (w + sigma): a periodic image X0 +- L of a wrapped coordinate
  // X0 in [-L/2, L/2) lies outside (-sigma, w + sigma), so only the
  // unshifted image can enter a frame
  int single_image;
  // candidate bins across the chain axis: the frame's extent w + 2 sigma
  // along each perpendicular axis is cut into nbin bins of side
  // >= sigma (1 + 2^-12); a sphere the mover can hit (|dp|, |dq| < sigma)
  // then lies in the mover's bin or a neighbour on both axes, also after
  // the FP32 rounding of the coordinates the bin index is computed from
  int nbin;
  float inv_hb;          // 1 / bin side
  int replay;            // replay periodic rattles (results unchanged)
};

struct State3 {
  int64_t t;
  int axis;
  int perm[8];
  double s[3];
};

struct Cell3 {
  double sum_b;
  int events, lifts, frozen, walls, chains, n_mem, replayed;
};

struct Totals3 {
  double sum_b, sum_disp, sum_b_w, sum_disp_w;
  long long sweeps, chains, events, lifts, frozen, walls, replayed;
};

// Legs of the current chain kept for the replay of periodic rattles (a
// power of two: the ring index is the leg number's low bits)
constexpr int kHist3 = 16;

// ---- kernels ----------------------------------------------------------------

__global__ void k3_begin(Geom3 g, State3* st, unsigned* sched) {
  if (threadIdx.x != 0) return;
  // persistent sweep: the work list from the start, a new epoch, no abort
  sched[0] = 0u;
  sched[1] += 1u;
  sched[2] = 0u;
  State3 s = *st;
  const U64x4 u = philox((uint64_t)s.t, ecmc::kPurposeSweep, 0, 0, g.seed, g.replica);
  for (int a = 0; a < 3; ++a) s.s[a] = unit_double(u.v[a]) * g.w;
  // colour order: permutation number floor(u3 * 8! / 2^64) of 0..7 in
  // lexicographic order, decoded from its factorial-base digits
  int code = (int)below_n(u.v[3], 40320);
  int pool[8] = {0, 1, 2, 3, 4, 5, 6, 7};
  const int radix[8] = {5040, 720, 120, 24, 6, 2, 1, 1};
  int left = 8;
  for (int i = 0; i < 8; ++i) {
    const int d = code / radix[i];
    code -= d * radix[i];
    s.perm[i] = pool[d];
    for (int j = d; j < left - 1; ++j) pool[j] = pool[j + 1];
    --left;
  }
  s.axis = (int)(s.t % 3);
  *st = s;
}

__global__ void k3_bin(Geom3 g, const State3* __restrict__ st, const double* __restrict__ px,
                       const double* __restrict__ py, const double* __restrict__ pz,
                       int* __restrict__ cnt, int* __restrict__ ids, int* __restrict__ cell_of,
                       int* err) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.N) return;
  const State3 s = *st;
  const int cx = cell_1d(px[i], s.s[0], g.L, g.inv_w, g.cells);
  const int cy = cell_1d(py[i], s.s[1], g.L, g.inv_w, g.cells);
  const int cz = cell_1d(pz[i], s.s[2], g.L, g.inv_w, g.cells);
  const int c = (cz * g.cells + cy) * g.cells + cx;
  cell_of[i] = c;
  const int slot = atomicAdd(&cnt[c], 1);
  if (slot < g.cap_mem) ids[(int64_t)c * g.cap_mem + slot] = (int)i;
  else atomicCAS(err, kOk, kCapacity);
}

// (s, key) before (bs, bk) for hit distances s, bs >= +0 (or +inf): the
// bit patterns compare like the values
__device__ __forceinline__ bool first_before(double s, long long k, double bs, long long bk) {
  return lt_nn(s, bs) || (dbits(s) == dbits(bs) && k < bk);
}

// Cold paths of cell3, kept out of line so that the hot loop's code stays
// small.  Every periodic image of the offset (x0, x1, x2) whose centre lies
// in the open slab (lo, hi)^3 (boxes below the single-image size): bit
// img = (kx+1)*9 + (ky+1)*3 + (kz+1).
__device__ __noinline__ unsigned images_mask3(double x0, double x1, double x2, double L,
                                              double lo, double hi) {
  unsigned mask = 0u;
  for (int kx = -1; kx <= 1; ++kx) {
    const double X = x0 + (double)kx * L;
    if (!(X > lo && X < hi)) continue;
    for (int ky = -1; ky <= 1; ++ky) {
      const double Y = x1 + (double)ky * L;
      if (!(Y > lo && Y < hi)) continue;
      for (int kz = -1; kz <= 1; ++kz) {
        const double Z = x2 + (double)kz * L;
        if (!(Z > lo && Z < hi)) continue;
        mask |= 1u << ((kx + 1) * 9 + (ky + 1) * 3 + (kz + 1));
      }
    }
  }
  return mask;
}

// A lane's best candidate: hit distance, b, tie-break key, frame index.
struct Hit3 {
  double s, b;
  long long k;
  int j;
};

// The warp's first hit by (s, key) through a shuffle tree, for keys that do
// not fit 32 bits (N >= 2^32 / 27).
__device__ __noinline__ Hit3 first_hit_tree(Hit3 h) {
#pragma unroll 1
  for (int off = 16; off > 0; off >>= 1) {
    const double os = __shfl_xor_sync(0xffffffffu, h.s, off);
    const double ob = __shfl_xor_sync(0xffffffffu, h.b, off);
    const long long ok2 = __shfl_xor_sync(0xffffffffu, h.k, off);
    const int oj = __shfl_xor_sync(0xffffffffu, h.j, off);
    if (first_before(os, ok2, h.s, h.k)) {
      h.s = os;
      h.b = ob;
      h.k = ok2;
      h.j = oj;
    }
  }
  return h;
}

// The distinct neighbour cells with two cells per side, where the cells at
// offsets -1 and +1 coincide (lane 0 only).
__device__ __noinline__ void neighbour_list_small(int* nbl, int cx, int cy, int cz, int nc, int c) {
  int n = 0;
  for (int dz = -1; dz <= 1; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        const int qx = (cx + dx + nc) % nc, qy = (cy + dy + nc) % nc, qz = (cz + dz + nc) % nc;
        const int q = (qz * nc + qy) * nc + qx;
        if (q == c) continue;
        bool dup = false;
        for (int e = 0; e < n; ++e) dup |= nbl[e] == q;
        if (!dup) nbl[n++] = q;
      }
  nbl[26] = n;
}

// Position loads: through L1 in the per-phase kernels (the writers finished
// in an earlier launch), from L2 in the persistent kernel (the writers may
// be warps of other SMs in the same launch).
template <bool CG>
__device__ __forceinline__ double ldpos(const double* p) {
  if constexpr (CG) return __ldcg(p);
  else return *p;
}

// One active cell of colour phase colour_index, by one warp: frame, chains,
// write-back, cell statistics.  base: the warp's shared memory.
template <bool CG>
__device__ __forceinline__ void cell3(const Geom3& g, const State3& st, int colour_index, int a,
                                      unsigned char* base, double* __restrict__ px,
                                      double* __restrict__ py, double* __restrict__ pz,
                                      const int* __restrict__ cnt, const int* __restrict__ ids,
                                      Cell3* __restrict__ cs, int* __restrict__ recs, int* err) {
  constexpr unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int colour = st.perm[colour_index];
  const int hx = g.cells >> 1, nc = g.cells;
  const int cx = 2 * (a % hx) + (colour & 1);
  const int cy = 2 * ((a / hx) % hx) + ((colour >> 1) & 1);
  const int cz = 2 * (a / (hx * hx)) + (colour >> 2);
  const int c = (cz * nc + cy) * nc + cx;
  const double L = g.L, w = g.w;
  const double o[3] = {st.s[0] + (double)cx * w, st.s[1] + (double)cy * w,
                       st.s[2] + (double)cz * w};

  double* C[3];
  C[0] = reinterpret_cast<double*>(base);
  C[1] = C[0] + g.cap_obj;
  C[2] = C[1] + g.cap_obj;
  long long* key = reinterpret_cast<long long*>(C[2] + g.cap_obj);
  // the chain's last kHist3 legs: start and end coordinate of the active
  // sphere along the axis, length, contact term bb - bs
  double* hP = reinterpret_cast<double*>(key + g.cap_obj);
  double* hE = hP + kHist3;
  double* hS = hE + kHist3;
  double* hT = hS + kHist3;
  float* F[3];  // FP32 roundings of C, kept current as members move
  F[0] = reinterpret_cast<float*>(hT + kHist3);
  F[1] = F[0] + g.cap_obj;
  F[2] = F[1] + g.cap_obj;
  int* sid = reinterpret_cast<int*>(F[2] + g.cap_obj);  // members sorted by id
  int* raw = sid + g.cap_mem;                           // members as bucketed
  int* nbl = raw + g.cap_mem;                           // 26 neighbour cells + count
  int* npre = nbl + 28;                                 // their bucket sizes, prefix sums
  int* hM = npre + 28;    // legs: active sphere, direction, kind (0 lift, 1 frozen, 2 wall)
  int* hSg = hM + kHist3;
  int* hK = hSg + kHist3;
  int* cand = hK + kHist3;                              // FP32 screen survivors
  int* ord = cand + g.cap_obj;                          // objects sorted by bin
  const int nb = g.nbin, nb2 = nb * nb;
  int* bst = ord + g.cap_obj;                           // bin starts, nb2 + 1
  int* cur = bst + nb2 + 1;                             // scatter cursors, nb2
  unsigned char* touched = reinterpret_cast<unsigned char*>(cur + nb2);

  const int nmem = min(cnt[c], g.cap_mem);
  for (int k = lane; k < nmem; k += 32) raw[k] = ids[(int64_t)c * g.cap_mem + k];
  if (nc >= 3) {
    // 26 distinct neighbour cells: lane e takes offset e of the 3x3x3 block
    // in (dz, dy, dx) order, the centre skipped
    if (lane < 26) {
      const int e = lane < 13 ? lane : lane + 1;
      int qx = cx + e % 3 - 1, qy = cy + (e / 3) % 3 - 1, qz = cz + e / 9 - 1;
      qx = qx < 0 ? qx + nc : (qx >= nc ? qx - nc : qx);
      qy = qy < 0 ? qy + nc : (qy >= nc ? qy - nc : qy);
      qz = qz < 0 ? qz + nc : (qz >= nc ? qz - nc : qz);
      nbl[lane] = (qz * nc + qy) * nc + qx;
    }
    if (lane == 0) nbl[26] = 26;
  } else if (lane == 0) {
    neighbour_list_small(nbl, cx, cy, cz, nc, c);
  }
  __syncwarp();
  // the neighbours' objects as one list: npre[e] = sum of the bucket sizes
  // of neighbours 0 .. e-1
  const int nnb = nbl[26];
  {
    const int nq = lane < nnb ? min(cnt[nbl[lane]], g.cap_mem) : 0;
    int incl = nq;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int v = __shfl_up_sync(FULL, incl, off);
      if (lane >= off) incl += v;
    }
    if (lane == 0) npre[0] = 0;
    if (lane < nnb) npre[lane + 1] = incl;
  }
  // members in ascending id (the rank of each is the number of smaller
  // ids); the positions are loaded before the rank is counted
  const double hL = 0.5 * L;
  for (int k = lane; k < nmem; k += 32) {
    const int v = raw[k];
    const double mx = ldpos<CG>(px + v), my = ldpos<CG>(py + v), mz = ldpos<CG>(pz + v);
    int r = 0;
    for (int j = 0; j < nmem; ++j) r += raw[j] < v ? 1 : 0;
    sid[r] = v;
    touched[r] = 0;
    C[0][r] = wrap_half_i(mx - o[0], L, hL);
    C[1][r] = wrap_half_i(my - o[1], L, hL);
    C[2][r] = wrap_half_i(mz - o[2], L, hL);
    F[0][r] = to_float_trunc(C[0][r]);
    F[1][r] = to_float_trunc(C[1][r]);
    F[2][r] = to_float_trunc(C[2][r]);
    key[r] = (long long)v * 27 + 13;
  }
  __syncwarp();
  // frozen images, appended in the order (neighbour, bucket slot, image):
  // 32 entries of the neighbours' joint list per round, warp prefix sums
  int nobj = nmem;
  const double lo = -g.sigma, hi = w + g.sigma;
  const int ntot = npre[nnb];
  // the bucket slot of entry t of the joint list (t < ntot)
  auto slot_of = [&](int t) {
    int el = 0, eh = nnb;  // the neighbour e with npre[e] <= t < npre[e + 1]
    while (eh - el > 1) {
      const int mid = (el + eh) >> 1;
      if (npre[mid] <= t) el = mid;
      else eh = mid;
    }
    return (int64_t)nbl[el] * g.cap_mem + (t - npre[el]);
  };
  // one round: the entries of 32 lanes (valid where in) with their box
  // positions p, appended as frame objects in lane order
  auto append = [&](bool in, int id, const double* p) {
    double X0[3] = {0.0, 0.0, 0.0};
    unsigned mask = 0u;  // bit img = (kx+1)*9 + (ky+1)*3 + (kz+1)
    if (in) {
      X0[0] = wrap_half_i(p[0] - o[0], L, hL);
      X0[1] = wrap_half_i(p[1] - o[1], L, hL);
      X0[2] = wrap_half_i(p[2] - o[2], L, hL);
      if (g.single_image) {
        if (dlt(lo, X0[0]) && dlt(X0[0], hi) && dlt(lo, X0[1]) && dlt(X0[1], hi) &&
            dlt(lo, X0[2]) && dlt(X0[2], hi))
          mask = 1u << 13;
      } else {
        mask = images_mask3(X0[0], X0[1], X0[2], L, lo, hi);
      }
    }
    const int nimg = __popc(mask);
    int incl = nimg;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int v = __shfl_up_sync(FULL, incl, off);
      if (lane >= off) incl += v;
    }
    int slot = nobj + incl - nimg;
    while (mask) {
      const int img = __ffs(mask) - 1;
      mask &= mask - 1;
      if (slot < g.cap_obj) {
        // X0 + k L for k in {-1, 0, 1}: (double)k * L is -L, +0.0 or L
        // exactly, and adding +0.0 only turns -0.0 into +0.0
        const int kx = img / 9 - 1, ky = (img / 3) % 3 - 1, kz = img % 3 - 1;
        C[0][slot] = kx == 0 ? plus_zero(X0[0]) : X0[0] + (kx > 0 ? L : -L);
        C[1][slot] = ky == 0 ? plus_zero(X0[1]) : X0[1] + (ky > 0 ? L : -L);
        C[2][slot] = kz == 0 ? plus_zero(X0[2]) : X0[2] + (kz > 0 ? L : -L);
        F[0][slot] = to_float_trunc(C[0][slot]);
        F[1][slot] = to_float_trunc(C[1][slot]);
        F[2][slot] = to_float_trunc(C[2][slot]);
        key[slot] = (long long)id * 27 + img;
      }
      ++slot;
    }
    nobj += __shfl_sync(FULL, incl, 31);
  };
  // two rounds per pass, their loads issued together so that the L2
  // latencies overlap
  for (int t0 = 0; t0 < ntot; t0 += 64) {
    const int ta = t0 + lane, tb = t0 + 32 + lane;
    const bool ina = ta < ntot, inb = tb < ntot;
    const int ida = ina ? ids[slot_of(ta)] : 0;
    const int idb = inb ? ids[slot_of(tb)] : 0;
    double pa[3] = {0.0, 0.0, 0.0}, pb[3] = {0.0, 0.0, 0.0};
    if (ina) {
      pa[0] = ldpos<CG>(px + ida);
      pa[1] = ldpos<CG>(py + ida);
      pa[2] = ldpos<CG>(pz + ida);
    }
    if (inb) {
      pb[0] = ldpos<CG>(px + idb);
      pb[1] = ldpos<CG>(py + idb);
      pb[2] = ldpos<CG>(pz + idb);
    }
    // one copy of the append code for both rounds
#pragma unroll 1
    for (int h = 0; h < 2; ++h) {
      if (h == 1 && t0 + 32 >= ntot) break;
      const double q[3] = {h ? pb[0] : pa[0], h ? pb[1] : pa[1], h ? pb[2] : pa[2]};
      append(h ? inb : ina, h ? idb : ida, q);
    }
  }
  const bool ok = nobj <= g.cap_obj;
  if (!ok && lane == 0) atomicCAS(err, kOk, kCapacity);
  __syncwarp();

  // bins across the sweep's axis (members move only along it, so the bins
  // hold for the whole phase): counting sort of the objects, q-major
  const int ax = st.axis, axp = ax == 0 ? 1 : 0, axq = ax == 2 ? 1 : 2;
  const float sigf = (float)g.sigma;
  auto bin_of = [&](float v) {
    const int b = (int)((v + sigf) * g.inv_hb);
    return b < 0 ? 0 : (b >= nb ? nb - 1 : b);
  };
  const int nobj_ok = ok ? nobj : 0;
  for (int i = lane; i <= nb2; i += 32) bst[i] = 0;
  __syncwarp();
  for (int o2 = lane; o2 < nobj_ok; o2 += 32)
    atomicAdd(&bst[1 + bin_of(F[axq][o2]) * nb + bin_of(F[axp][o2])], 1);
  __syncwarp();
  if (nb2 < 32) {
    // bin starts by a warp scan of the counts (bst[0] = 0)
    int v = lane <= nb2 ? bst[lane] : 0;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int u = __shfl_up_sync(FULL, v, off);
      if (lane >= off) v += u;
    }
    if (lane <= nb2) bst[lane] = v;
  } else if (lane == 0) {
    for (int i = 1; i <= nb2; ++i) bst[i] += bst[i - 1];
  }
  __syncwarp();
  for (int i = lane; i < nb2; i += 32) cur[i] = bst[i];
  __syncwarp();
  for (int o2 = lane; o2 < nobj_ok; o2 += 32)
    ord[atomicAdd(&cur[bin_of(F[axq][o2]) * nb + bin_of(F[axp][o2])], 1)] = o2;
  __syncwarp();

  // the cell's chains
  double* CA = C[ax];
  double* CP = C[axp];
  double* CQ = C[axq];
  float* FA = F[ax];
  const float* FP = F[axp];
  const float* FQ = F[axq];
  const double INF = __longlong_as_double(0x7ff0000000000000ll);
  // keys id * 27 + image below 2^32 - 1: the reduction below may use 32-bit minima
  const bool key32 = g.N * 27 < ((int64_t)1 << 32) - 27;
  double sum_b = 0.0;
  int n_ev = 0, n_li = 0, n_fr = 0, n_wa = 0, n_ch = 0, n_rep = 0;
  for (int k = 0; k < g.n_m; ++k) {
    int* rec = recs != nullptr ? recs + 4 * ((int64_t)c * g.n_m + k) : nullptr;
    if (!ok || nmem == 0) {
      if (rec != nullptr && lane == 0) {
        rec[0] = -1;
        rec[1] = -1;
        rec[2] = 0;
        rec[3] = 0;
      }
      continue;
    }
    const U64x4 v = philox((uint64_t)st.t, ecmc::kPurposeChain, (uint64_t)c, (uint64_t)k,
                           g.seed, g.replica);
    int m = (int)below_n(v.v[0], (uint64_t)nmem);
    int sg = (v.v[1] >> 63) ? -1 : 1;
    const int start_id = sid[m];
    double r = g.ell;
    int ch_ev = 0, ch_wa = 0;
    int n_leg = 0;        // legs recorded in the history
    int64_t ch_rep = 0;   // legs of this chain replayed
    if (lane == 0) touched[m] = 1;
    ++n_ch;
    for (int64_t iter = 0;; ++iter) {
      if (iter + ch_rep >= ecmc::kMaxEventsPerChain) {
        if (lane == 0) atomicCAS(err, kOk, kChainCap);
        break;
      }
      __syncwarp();
      const double P = CA[m], Pp = CP[m], Pq = CQ[m];
      const float P32 = FA[m], Pp32 = FP[m], Pq32 = FQ[m];
      const double sw = clamp0(sg > 0 ? w - P : P);
      double bs = INF, bb = 0.0;
      long long bk = LLONG_MAX;
      int bj = -1;
      // candidates: the three rows of bins around the mover, each a
      // contiguous run of ord[]; FP32 screen, survivors compacted into
      // cand[] so that the FP64 tests below take one warp-wide pass
      const int bpm = bin_of(Pp32), bqm = bin_of(Pq32);
      const int plo = bpm > 0 ? bpm - 1 : 0, phi = bpm < nb - 1 ? bpm + 1 : nb - 1;
      int rs[3], rl[3];
#pragma unroll
      for (int k3 = 0; k3 < 3; ++k3) {
        const int row = bqm - 1 + k3;
        const bool in = row >= 0 && row < nb;
        rs[k3] = in ? bst[row * nb + plo] : 0;
        rl[k3] = in ? bst[row * nb + phi + 1] - rs[k3] : 0;
      }
      const int n_c = rl[0] + rl[1] + rl[2];
      int ns = 0;
      for (int t0 = 0; t0 < n_c; t0 += 32) {
        const int t = t0 + lane;
        bool pass = false;
        int j = -1;
        if (t < n_c) {
          j = t < rl[0] ? ord[rs[0] + t]
                        : (t < rl[0] + rl[1] ? ord[rs[1] + t - rl[0]]
                                             : ord[rs[2] + t - rl[0] - rl[1]]);
        }
        if (t < n_c && j != m) {
          const float da32 = FA[j] - P32;
          const float dp32 = FP[j] - Pp32, dq32 = FQ[j] - Pq32;
          pass = ((sg > 0 ? da32 : -da32) > -g.scr_b) &&
                 (dp32 * dp32 + dq32 * dq32 < g.scr_c2);
        }
        const unsigned bal = __ballot_sync(FULL, pass);
        if (pass) cand[ns + __popc(bal & ((1u << lane) - 1u))] = j;
        ns += __popc(bal);
      }
      __syncwarp();
      for (int t = lane; t < ns; t += 32) {
        const int j = cand[t];
        const double da = CA[j] - P;
        const double b = flip_if(da, sg < 0);
        if (dbits(b) <= 0) continue;  // b > 0
        const double dp = CP[j] - Pp;
        const double dq = CQ[j] - Pq;
        const double c2 = dp * dp + dq * dq;
        if (!lt_nn(c2, g.sig2)) continue;
        // sigma^2 - c^2 is a positive normal number here (sigma in
        // [2^-40, 2^40]), as sqrt_rn requires
        const double s = clamp0(b - sqrt_rn(g.sig2 - c2));
        const long long kj = key[j];
        if (first_before(s, kj, bs, bk)) {
          bs = s;
          bb = b;
          bk = kj;
          bj = j;
        }
      }
      if (key32) {
        // the first hit by (s, key) with three hardware minima: s >= +0 (or
        // +inf) orders as its bit pattern, compared high word then low word,
        // and keys below 2^32 break exact ties; lanes without a candidate
        // hold (+inf, max key)
        const unsigned long long sb = (unsigned long long)dbits(bs);
        const unsigned hi = (unsigned)(sb >> 32), lo = (unsigned)sb;
        const unsigned mhi = __reduce_min_sync(FULL, hi);
        const unsigned mlo = __reduce_min_sync(FULL, hi == mhi ? lo : 0xffffffffu);
        const bool at = hi == mhi && lo == mlo;
        const unsigned k32 = bk == LLONG_MAX ? 0xffffffffu : (unsigned)bk;
        const unsigned mk = __reduce_min_sync(FULL, at ? k32 : 0xffffffffu);
        const int win = __ffs(__ballot_sync(FULL, at && k32 == mk)) - 1;
        bs = __shfl_sync(FULL, bs, win);
        bb = __shfl_sync(FULL, bb, win);
        bk = __shfl_sync(FULL, bk, win);
        bj = __shfl_sync(FULL, bj, win);
      } else {
        const Hit3 hw = first_hit_tree(Hit3{bs, bb, bk, bj});
        bs = hw.s;
        bb = hw.b;
        bk = hw.k;
        bj = hw.j;
      }
      __syncwarp();
      if (le_nn(r, bs) && le_nn(r, sw)) {  // budget used up
        if (lane == 0) {
          CA[m] = P + (sg > 0 ? r : -r);
          FA[m] = to_float_trunc(CA[m]);
        }
        break;
      }
      const int hi = n_leg & (kHist3 - 1);
      int kind;
      if (le_nn(bs, sw)) {  // contact
        // one FP64 addition gives three results: lane 0 the mover's new
        // coordinate P +- bs, lane 2 the contact term bb - bs (summed on
        // lane 2), every other lane the budget left, r - bs; x - y is by
        // definition x + (-y), so each equals its separate expression
        const double z = (lane == 0 ? P : (lane == 2 ? bb : r)) +
                         flip_if(bs, lane == 0 ? sg < 0 : true);
        kind = bj < nmem ? 0 : 1;
        if (lane == 0) {
          CA[m] = z;
          FA[m] = to_float_trunc(z);
          hP[hi] = P;
          hE[hi] = z;
          hS[hi] = bs;
          hM[hi] = m;
          hSg[hi] = sg;
          hK[hi] = kind;
        }
        if (lane == 2) {
          sum_b += z;
          hT[hi] = z;
        }
        r = __shfl_sync(FULL, z, 1);
        ++n_ev;
        ++ch_ev;
        if (kind == 0) {  // lift
          ++n_li;
          m = bj;
          if (lane == 0) touched[m] = 1;
        } else {  // frozen sphere: back along the axis
          sg = -sg;
          ++n_fr;
        }
      } else {  // wall: onto the wall, back along the axis
        kind = 2;
        if (lane == 0) {
          CA[m] = sg > 0 ? w : 0.0;
          FA[m] = to_float_trunc(CA[m]);
          hP[hi] = P;
          hE[hi] = CA[m];
          hS[hi] = sw;
          hM[hi] = m;
          hSg[hi] = sg;
          hK[hi] = 2;
        }
        r = r - sw;
        sg = -sg;
        ++n_wa;
        ++ch_wa;
      }
      ++n_leg;
      if (g.replay && kind != 0 && n_leg >= 2) {
        // Replay of a periodic rattle.  After a turn-back, lane l tests the
        // period K = 2 (l + 1) <= n_leg: the next leg starts from the state
        // (active sphere, direction, coordinate bit for bit) that leg
        // n_leg - K started from, and every sphere active in those K legs
        // is back at its coordinate at the start of its first of them.  Frozen spheres
        // and walls do not move, so the whole frame is then as it was K
        // legs ago and, the dynamics being deterministic with the budget
        // entering a leg only through its end, the following legs repeat
        // the recorded ones for as long as the budget exceeds their length.
        __syncwarp();
        bool per = false;
        if (lane < kHist3 / 2 && 2 * (lane + 1) <= n_leg) {
          const int K = 2 * (lane + 1);
          const int i0 = (n_leg - K) & (kHist3 - 1);
          if (hM[i0] == m && hSg[i0] == sg && dbits(hP[i0]) == dbits(CA[m])) {
            per = true;
            for (int j = 1; j < K; ++j) {
              const int ij = (n_leg - K + j) & (kHist3 - 1);
              const int d = hM[ij];
              bool first = true;
              for (int i = 0; i < j; ++i) first = first && hM[(n_leg - K + i) & (kHist3 - 1)] != d;
              if (first && dbits(CA[d]) != dbits(hP[ij])) per = false;
            }
          }
        }
        const unsigned pb = __ballot_sync(FULL, per);
        if (pb != 0u) {
          const int K = 2 * __ffs(pb), b0 = n_leg - K;
          int j = 0;
          for (;;) {  // whole legs while the budget exceeds them
            const int ij = (b0 + j) & (kHist3 - 1);
            const double st_j = hS[ij];
            if (le_nn(r, st_j) || iter + ch_rep + 1 >= ecmc::kMaxEventsPerChain) break;
            r = r - st_j;
            const int kd = hK[ij];
            if (kd == 2) {
              ++n_wa;
              ++ch_wa;
            } else {
              ++n_ev;
              ++ch_ev;
              if (kd == 0) ++n_li;
              else ++n_fr;
              if (lane == 2) sum_b += hT[ij];
            }
            ++ch_rep;
            ++n_rep;
            j = j + 1 == K ? 0 : j + 1;
          }
          // the frame is as at the start of leg b0 (and of every K legs
          // after it); the recorded legs b0 .. b0 + j - 1 bring it to the
          // start of the leg in which the budget runs out, which the full
          // search then takes
          if (lane == 0)
            for (int i = 0; i < j; ++i) {
              const int ii = (b0 + i) & (kHist3 - 1);
              CA[hM[ii]] = hE[ii];
              FA[hM[ii]] = to_float_trunc(hE[ii]);
            }
          m = hM[(b0 + j) & (kHist3 - 1)];
          sg = hSg[(b0 + j) & (kHist3 - 1)];
          n_leg = 0;
        }
      }
    }
    __syncwarp();
    if (rec != nullptr && lane == 0) {
      rec[0] = start_id;
      rec[1] = sid[m];
      rec[2] = ch_ev;
      rec[3] = ch_wa;
    }
  }
  __syncwarp();
  // members that moved, back in box coordinates
  for (int q = lane; q < nmem; q += 32) {
    if (!touched[q]) continue;
    const int i = sid[q];
    px[i] = wrap_box0(C[0][q] + o[0], L);
    py[i] = wrap_box0(C[1][q] + o[1], L);
    pz[i] = wrap_box0(C[2][q] + o[2], L);
  }
  sum_b = __shfl_sync(FULL, sum_b, 2);  // the contact sum is kept on lane 2
  if (lane == 0) {
    Cell3 s;
    s.sum_b = sum_b;
    s.events = n_ev;
    s.lifts = n_li;
    s.frozen = n_fr;
    s.walls = n_wa;
    s.chains = n_ch;
    s.n_mem = nmem;
    s.replayed = n_rep;
    cs[c] = s;
  }
}

__global__ void __launch_bounds__(32 * kWarpsMax) k3_phase(
    Geom3 g, const State3* __restrict__ stp, int colour_index, double* __restrict__ px,
    double* __restrict__ py, double* __restrict__ pz, const int* __restrict__ cnt,
    const int* __restrict__ ids, Cell3* __restrict__ cs, int* __restrict__ recs, int* err) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int warp = threadIdx.x >> 5;
  const int a = blockIdx.x * (blockDim.x >> 5) + warp;
  if (a >= g.nact) return;  // warp-uniform
  const State3 st = *stp;
  cell3<false>(g, st, colour_index, a, smem + (size_t)warp * g.warp_bytes, px, py, pz, cnt, ids,
               cs, recs, err);
}

__device__ __forceinline__ unsigned long long global_ns3() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned load_volatile3(const unsigned* p) {
  return *(const volatile unsigned*)p;
}

// The persistent sweep: all eight colour phases in one launch.  Work item
// i = ci * nact + a (colour phase ci, active cell a) is taken from a device
// counter; the warp waits until each of the cell's 26 neighbours whose colour
// comes earlier in this sweep's order has finished (done[] holds the sweep's
// epoch), then processes the cell and publishes it.  A cell of a later
// colour has not moved yet and waits for this one in turn, so the result is
// that of the per-phase launches bit for bit.  Progress: an item waits only
// for smaller items, taken earlier by running warps that wait only for still
// smaller ones.  Every wait is bounded (global timer): on timeout the kernel
// raises kWaitTimeout and an abort flag that makes every warp leave.
__global__ void __launch_bounds__(32 * kWarpsMax) k3_sweep(
    Geom3 g, const State3* __restrict__ stp, double* __restrict__ px, double* __restrict__ py,
    double* __restrict__ pz, const int* __restrict__ cnt, const int* __restrict__ ids,
    Cell3* __restrict__ cs, int* __restrict__ recs, unsigned* sched, unsigned* done,
    unsigned long long wait_ns, int wait_test, int* err) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr unsigned FULL = 0xffffffffu;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned char* base = smem + (size_t)warp * g.warp_bytes;
  const State3 st = *stp;
  const unsigned epoch = load_volatile3(&sched[1]);
  // the failure test waits for a value nobody writes
  const unsigned want = wait_test ? (epoch ^ 0x80000000u) : epoch;
  int phase_of[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) phase_of[st.perm[k]] = k;
  const int n_items = 8 * g.nact, hx = g.cells >> 1, nc = g.cells;
  for (;;) {
    int item = 0;
    if (lane == 0) item = (int)atomicAdd(&sched[0], 1u);
    item = __shfl_sync(FULL, item, 0);
    if (item >= n_items || load_volatile3(&sched[2]) != 0u) break;
    const int ci = item / g.nact, a = item - ci * g.nact;
    const int colour = st.perm[ci];
    const int cx = 2 * (a % hx) + (colour & 1);
    const int cy = 2 * ((a / hx) % hx) + ((colour >> 1) & 1);
    const int cz = 2 * (a / (hx * hx)) + (colour >> 2);
    bool ok = true;
    if (ci > 0 && lane < 26) {
      // lane d waits for neighbour d of the 3x3x3 block (the centre skipped)
      const int e = lane < 13 ? lane : lane + 1;
      const int dx = e % 3 - 1, dy = (e / 3) % 3 - 1, dz = e / 9 - 1;
      const int ncol = colour ^ (dx != 0 ? 1 : 0) ^ (dy != 0 ? 2 : 0) ^ (dz != 0 ? 4 : 0);
      if (phase_of[ncol] < ci) {
        const int q = (((cz + dz + nc) % nc) * nc + (cy + dy + nc) % nc) * nc + (cx + dx + nc) % nc;
        if (load_volatile3(&done[q]) != want) {
          const unsigned long long t0 = global_ns3();
          while (load_volatile3(&done[q]) != want) {
            if (load_volatile3(&sched[2]) != 0u) {
              ok = false;
              break;
            }
            if (global_ns3() - t0 > wait_ns) {
              atomicCAS(err, kOk, kWaitTimeout);
              atomicExch(&sched[2], 1u);
              ok = false;
              break;
            }
            __nanosleep(256);
          }
        }
      }
    }
    if (!__all_sync(FULL, ok)) break;
    __threadfence();  // the finished neighbours' positions are visible from here on
    cell3<true>(g, st, ci, a, base, px, py, pz, cnt, ids, cs, recs, err);
    __syncwarp();
    if (lane == 0) {
      __threadfence();
      *(volatile unsigned*)&done[(cz * nc + cy) * nc + cx] = epoch;
    }
    __syncwarp();
  }
}

// End of sweep (one block of 256): the cells' sums in a fixed order, the
// running totals, the sweep's member-weighted pressure sums, t + 1.
__global__ void __launch_bounds__(256) k3_end(Geom3 g, State3* st, const Cell3* __restrict__ cs,
                                             Totals3* tot, double* history, int64_t* hist_len) {
  __shared__ double sd[2][8];
  __shared__ long long sl[6][8];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  double b = 0.0, bw = 0.0;
  long long v[6] = {0, 0, 0, 0, 0, 0};
  for (int c = tid; c < g.ncell; c += 256) {
    const Cell3 s = cs[c];
    b += s.sum_b;
    bw += (double)s.n_mem * s.sum_b;
    v[0] += s.events;
    v[1] += s.lifts;
    v[2] += s.frozen;
    v[3] += s.walls;
    v[4] += s.chains;
    v[5] += s.replayed;
  }
  for (int off = 16; off > 0; off >>= 1) {
    b += __shfl_down_sync(0xffffffffu, b, off);
    bw += __shfl_down_sync(0xffffffffu, bw, off);
    for (int q = 0; q < 6; ++q) v[q] += __shfl_down_sync(0xffffffffu, v[q], off);
  }
  if (lane == 0) {
    sd[0][wid] = b;
    sd[1][wid] = bw;
    for (int q = 0; q < 6; ++q) sl[q][wid] = v[q];
  }
  __syncthreads();
  if (tid != 0) return;
  double B = 0.0, BW = 0.0;
  long long V[6] = {0, 0, 0, 0, 0, 0};
  for (int wv = 0; wv < 8; ++wv) {
    B += sd[0][wv];
    BW += sd[1][wv];
    for (int q = 0; q < 6; ++q) V[q] += sl[q][wv];
  }
  const double dw = (double)g.N * (double)g.n_m * g.ell;
  Totals3& T = *tot;
  T.sum_b += B;
  T.sum_b_w += BW;
  T.sum_disp += (double)V[4] * g.ell;
  T.sum_disp_w += dw;
  T.events += V[0];
  T.lifts += V[1];
  T.frozen += V[2];
  T.walls += V[3];
  T.chains += V[4];
  T.replayed += V[5];
  T.sweeps += 1;
  const int64_t n = *hist_len;
  if (n < kHistoryCap) {
    history[2 * n] = BW;
    history[2 * n + 1] = dw;
  }
  *hist_len = n + 1;
  st->t += 1;
}

// interleaved [x0, y0, z0, ...] <-> three arrays
__global__ void k3_split(const double* __restrict__ xyz, int64_t N, double* __restrict__ px,
                         double* __restrict__ py, double* __restrict__ pz) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  px[i] = xyz[3 * i];
  py[i] = xyz[3 * i + 1];
  pz[i] = xyz[3 * i + 2];
}

__global__ void k3_join(const double* __restrict__ px, const double* __restrict__ py,
                        const double* __restrict__ pz, int64_t N, double* __restrict__ xyz) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  xyz[3 * i] = px[i];
  xyz[3 * i + 1] = py[i];
  xyz[3 * i + 2] = pz[i];
}

// Smallest squared minimum-image distance below rcut^2 over the pairs of the
// last binning's 27-cell neighbourhoods (FP64, the oracle's formula), as the
// bits of a non-negative double (their order is the order of the values).
__global__ void k3_min_dist(Geom3 g, const double* __restrict__ px, const double* __restrict__ py,
                            const double* __restrict__ pz, const int* __restrict__ cnt,
                            const int* __restrict__ ids, const int* __restrict__ cell_of,
                            unsigned long long r2_bits, unsigned long long* out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long best = r2_bits;
  if (i < g.N) {
    const int c = cell_of[i], nc = g.cells;
    const int cx = c % nc, cy = (c / nc) % nc, cz = c / (nc * nc);
    const double xi = px[i], yi = py[i], zi = pz[i];
    for (int dz = -1; dz <= 1; ++dz)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          const int q = (((cz + dz + nc) % nc) * nc + (cy + dy + nc) % nc) * nc +
                        (cx + dx + nc) % nc;
          const int nq = min(cnt[q], g.cap_mem);
          for (int k = 0; k < nq; ++k) {
            const int j = ids[(int64_t)q * g.cap_mem + k];
            if (j == i) continue;
            const double ex = wrap_half(px[j] - xi, g.L);
            const double ey = wrap_half(py[j] - yi, g.L);
            const double ez = wrap_half(pz[j] - zi, g.L);
            const double d2 = ex * ex + ey * ey + ez * ez;
            const unsigned long long bits = __double_as_longlong(d2);
            best = bits < best ? bits : best;
          }
        }
  }
  for (int off = 16; off > 0; off >>= 1) {
    const unsigned long long o2 = __shfl_xor_sync(0xffffffffu, best, off);
    best = o2 < best ? o2 : best;
  }
  if ((threadIdx.x & 31) == 0 && best < r2_bits) atomicMin(out, best);
}

}  // namespace ecmc3

// ---- host side ----------------------------------------------------------------

using namespace ecmc3;

struct ecmc3_ctx {
  Geom3 g;
  cudaStream_t stream = nullptr, own = nullptr;
  double *px = nullptr, *py = nullptr, *pz = nullptr, *xyz_tmp = nullptr;
  int *cnt = nullptr, *ids = nullptr, *cell_of = nullptr, *err = nullptr, *recs = nullptr;
  unsigned *sched = nullptr, *done = nullptr;  // persistent sweep: work counter, epoch, abort
  int persistent = 1, fused_blocks = 0;
  unsigned long long wait_ns = 5000000000ull;
  int wait_test = 0;
  Cell3* cs = nullptr;
  State3* st = nullptr;
  Totals3* tot = nullptr;
  double* history = nullptr;
  int64_t* hist_len = nullptr;
  unsigned long long* u64 = nullptr;
  int warps = 1;
  int64_t t_host = 0;
  bool valid = false;
};

namespace {

int fail3(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  return ecmc::report_error(code, buf);
}

#define CK3(call)                                                                         \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return fail3(e_ == cudaErrorMemoryAllocation ? ECMC_ERR_OOM : ECMC_ERR_CUDA,        \
                   "%s failed: %s", #call, cudaGetErrorString(e_));                       \
  } while (0)

// spheres of diameter sigma whose centres lie in a cube of side s: they sit
// inside the cube of side s + sigma, and no packing of spheres is denser
// than pi / (3 sqrt 2), so there are at most sqrt(2) (s + sigma)^3 / sigma^3
int sphere_bound(double s, double sigma) {
  const double q = (s + sigma) / sigma;
  return (int)std::floor(std::sqrt(2.0) * q * q * q) + 2;
}

int check3(ecmc3_ctx* h) {
  int e = 0;
  CK3(cudaMemcpyAsync(&e, h->err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CK3(cudaStreamSynchronize(h->stream));
  if (e == kCapacity) {
    h->valid = false;
    return fail3(ECMC_ERR_CAPACITY, "a cell bucket or frame exceeded its packing bound");
  }
  if (e == kChainCap) {
    h->valid = false;
    return fail3(ECMC_ERR_CHAIN_CAP, "a chain reached the per-chain event cap");
  }
  if (e == kWaitTimeout) {
    h->valid = false;
    CK3(cudaMemsetAsync(h->err, 0, sizeof(int), h->stream));
    return fail3(ECMC_ERR_TIMEOUT, "a dependency wait of the persistent sweep exceeded %.0f ms; "
                 "the sweep was abandoned (positions must be set again)",
                 (double)h->wait_ns * 1e-6);
  }
  return ECMC_OK;
}

int enqueue_sweep(ecmc3_ctx* h, bool records) {
  const Geom3& g = h->g;
  CK3(cudaMemsetAsync(h->cnt, 0, sizeof(int) * (size_t)g.ncell, h->stream));
  k3_begin<<<1, 32, 0, h->stream>>>(g, h->st, h->sched);
  k3_bin<<<(unsigned)((g.N + 255) / 256), 256, 0, h->stream>>>(g, h->st, h->px, h->py, h->pz,
                                                               h->cnt, h->ids, h->cell_of,
                                                               h->err);
  const int wpb = h->warps;
  const size_t sm = (size_t)wpb * g.warp_bytes;
  if (h->persistent && h->fused_blocks > 0) {
    k3_sweep<<<(unsigned)h->fused_blocks, 32 * wpb, sm, h->stream>>>(
        g, h->st, h->px, h->py, h->pz, h->cnt, h->ids, h->cs, records ? h->recs : nullptr,
        h->sched, h->done, h->wait_ns, h->wait_test, h->err);
  } else {
    const unsigned blocks = (unsigned)((g.nact + wpb - 1) / wpb);
    for (int ci = 0; ci < 8; ++ci)
      k3_phase<<<blocks, 32 * wpb, sm, h->stream>>>(g, h->st, ci, h->px, h->py, h->pz, h->cnt,
                                                    h->ids, h->cs, records ? h->recs : nullptr,
                                                    h->err);
  }
  k3_end<<<1, 256, 0, h->stream>>>(g, h->st, h->cs, h->tot, h->history, h->hist_len);
  CK3(cudaGetLastError());
  return ECMC_OK;
}

int bin_now(ecmc3_ctx* h) {
  const Geom3& g = h->g;
  CK3(cudaMemsetAsync(h->cnt, 0, sizeof(int) * (size_t)g.ncell, h->stream));
  k3_begin<<<1, 32, 0, h->stream>>>(g, h->st, h->sched);
  k3_bin<<<(unsigned)((g.N + 255) / 256), 256, 0, h->stream>>>(g, h->st, h->px, h->py, h->pz,
                                                               h->cnt, h->ids, h->cell_of,
                                                               h->err);
  CK3(cudaGetLastError());
  return ECMC_OK;
}

double rcut3(const Geom3& g) { return std::fmin(2.0 * g.sigma, g.w); }

int min_dist2_3(ecmc3_ctx* h, double* d2) {
  const Geom3& g = h->g;
  const double rc = rcut3(g), r2 = rc * rc;
  unsigned long long bits = 0;
  std::memcpy(&bits, &r2, sizeof(r2));
  CK3(cudaMemcpyAsync(h->u64, &bits, sizeof(bits), cudaMemcpyHostToDevice, h->stream));
  k3_min_dist<<<(unsigned)((g.N + 255) / 256), 256, 0, h->stream>>>(
      g, h->px, h->py, h->pz, h->cnt, h->ids, h->cell_of, bits, h->u64);
  CK3(cudaGetLastError());
  CK3(cudaMemcpyAsync(&bits, h->u64, sizeof(bits), cudaMemcpyDeviceToHost, h->stream));
  const int rc2 = check3(h);
  if (rc2) return rc2;
  std::memcpy(d2, &bits, sizeof(*d2));
  return ECMC_OK;
}

int load_dev(ecmc3_ctx* h, const double* xyz_dev, int64_t t0) {
  const Geom3& g = h->g;
  k3_split<<<(unsigned)((g.N + 255) / 256), 256, 0, h->stream>>>(xyz_dev, g.N, h->px, h->py,
                                                                 h->pz);
  State3 s;
  std::memset(&s, 0, sizeof(s));
  s.t = t0;
  CK3(cudaMemcpyAsync(h->st, &s, sizeof(s), cudaMemcpyHostToDevice, h->stream));
  CK3(cudaMemsetAsync(h->tot, 0, sizeof(Totals3), h->stream));
  CK3(cudaMemsetAsync(h->hist_len, 0, sizeof(int64_t), h->stream));
  CK3(cudaMemsetAsync(h->err, 0, sizeof(int), h->stream));
  h->t_host = t0;
  h->valid = true;
  int rc = bin_now(h);
  if (rc) return rc;
  rc = check3(h);
  if (rc) return rc;
  double d2 = 0.0;
  rc = min_dist2_3(h, &d2);
  if (rc) return rc;
  if (d2 < g.sig2 * (1.0 - 1e-9)) {
    h->valid = false;
    return fail3(ECMC_ERR_OVERLAP, "positions overlap: smallest distance %.17g < sigma",
                 std::sqrt(d2));
  }
  return ECMC_OK;
}

void free3(ecmc3_ctx* h) {
  cudaFree(h->px);
  cudaFree(h->py);
  cudaFree(h->pz);
  cudaFree(h->xyz_tmp);
  cudaFree(h->cnt);
  cudaFree(h->ids);
  cudaFree(h->cell_of);
  cudaFree(h->err);
  cudaFree(h->recs);
  cudaFree(h->cs);
  cudaFree(h->st);
  cudaFree(h->tot);
  cudaFree(h->history);
  cudaFree(h->hist_len);
  cudaFree(h->u64);
  cudaFree(h->sched);
  cudaFree(h->done);
  if (h->own) cudaStreamDestroy(h->own);
}

// shared memory of one warp's frame, and the launch's warps per block
int layout3(ecmc3_ctx* h) {
  Geom3& g = h->g;
  g.warp_bytes = (int)(((size_t)g.cap_obj * (3 * sizeof(double) + sizeof(long long) +
                                             3 * sizeof(float) + 2 * sizeof(int)) +
                        (size_t)(2 * g.nbin * g.nbin + 1) * sizeof(int) +
                        (size_t)g.cap_mem * 2 * sizeof(int) + 56 * sizeof(int) +
                        (size_t)kHist3 * (4 * sizeof(double) + 3 * sizeof(int)) +
                        (size_t)g.cap_mem + 15) &
                       ~(size_t)15);
  int dev = 0, optin = 0, n_sm = 0;
  CK3(cudaGetDevice(&dev));
  CK3(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  CK3(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
  if ((size_t)g.warp_bytes > (size_t)optin)
    return fail3(ECMC_ERR_UNSUPPORTED, "a cell's frame (%d bytes) exceeds shared memory",
                 g.warp_bytes);
  // The attribute is per kernel for the whole process: request the most the
  // kernels can have, so that a handle with small frames never lowers the
  // limit a handle with larger frames launches with.
  cudaFuncAttributes fa;
  CK3(cudaFuncGetAttributes(&fa, k3_phase));
  CK3(cudaFuncSetAttribute(k3_phase, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           optin - (int)fa.sharedSizeBytes));
  CK3(cudaFuncGetAttributes(&fa, k3_sweep));
  CK3(cudaFuncSetAttribute(k3_sweep, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           optin - (int)fa.sharedSizeBytes));
  // block shape: the warps per block (one cell each) that keep the most
  // cells resident per SM; larger blocks on ties
  int wpb = 1, per_sm = 0, best = -1;
  for (int w = 1; w <= kWarpsMax; ++w) {
    const size_t smw = (size_t)w * g.warp_bytes;
    if (smw > (size_t)optin) break;
    int nb = 0;
    CK3(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k3_sweep, 32 * w, smw));
    if (nb * w >= best) {
      best = nb * w;
      wpb = w;
      per_sm = nb;
    }
  }
  h->warps = wpb;
  // the persistent grid: as many blocks as are resident at once, at most one
  // warp per work item
  const long long items = 8LL * g.nact;
  long long blocks = (long long)per_sm * n_sm;
  if (blocks > (items + wpb - 1) / wpb) blocks = (items + wpb - 1) / wpb;
  h->fused_blocks = per_sm > 0 ? (int)blocks : 0;
  return ECMC_OK;
}

}  // namespace

extern "C" {

int ecmc3_create(ecmc3_t* out, int64_t N, double L, double sigma, int cells, double ell,
                 uint64_t seed) {
  if (!out) return fail3(ECMC_ERR_ARG, "NULL output handle");
  *out = nullptr;
  if (N < 1 || N >= (int64_t(1) << 30)) return fail3(ECMC_ERR_ARG, "N out of range");
  int64_t k = (int64_t)std::llround(std::cbrt((double)N));
  while (k * k * k > N) --k;
  while ((k + 1) * (k + 1) * (k + 1) <= N) ++k;
  if (k * k * k != N) return fail3(ECMC_ERR_ARG, "N must be a perfect cube (lattice start)");
  if (!(L > 0.0) || !(sigma > 0.0) || !std::isfinite(L) || !std::isfinite(sigma))
    return fail3(ECMC_ERR_ARG, "L and sigma must be positive");
  if (!(sigma >= std::ldexp(1.0, -40) && sigma <= std::ldexp(1.0, 40) &&
        L < std::ldexp(sigma, 40)))
    return fail3(ECMC_ERR_ARG, "sigma must lie in [2^-40, 2^40] and L below 2^40 sigma");
  if (cells < 2 || (cells & 1) || cells > 1024)
    return fail3(ECMC_ERR_ARG, "cells per side must be even, >= 2 and <= 1024");
  if (!(L / (double)cells > sigma)) return fail3(ECMC_ERR_ARG, "cell side must exceed sigma");
  if (!(L / (double)k > sigma)) return fail3(ECMC_ERR_ARG, "cubic lattice would overlap");
  if (!(ell >= 0.0) || !std::isfinite(ell)) return fail3(ECMC_ERR_ARG, "ell must be >= 0");
  ecmc3_ctx* h = new ecmc3_ctx();
  Geom3& g = h->g;
  std::memset(&g, 0, sizeof(g));
  g.N = N;
  g.L = L;
  g.sigma = sigma;
  g.sig2 = sigma * sigma;
  g.cells = cells;
  g.ncell = cells * cells * cells;
  g.nact = g.ncell / 8;
  g.w = L / (double)cells;
  g.inv_w = 1.0 / g.w;
  g.ell = ell;
  g.n_m = 1;
  g.replay = 1;
  g.seed = seed;
  g.replica = 0;
  {
    const double M = g.w + 2.0 * sigma;
    const double d = 8.0 * std::ldexp(1.0, -24) * M;
    g.scr_b = (float)(2.0 * d);
    const double c2 = sigma * sigma + 4.0 * d * sigma + 2.0 * d * d +
                      4.0 * std::ldexp(1.0, -24) * (sigma * sigma + 4.0 * M * M);
    g.scr_c2 = std::nextafter((float)(sigma * sigma + 2.0 * (c2 - sigma * sigma)), 1e30f);
  }
  g.single_image = L >= 2.0 * (g.w + sigma) ? 1 : 0;
  {
    const double ext = g.w + 2.0 * sigma;
    int nb = (int)std::floor(ext / (sigma * (1.0 + std::ldexp(1.0, -12))));
    if (nb < 1) nb = 1;
    if (nb > 64) nb = 64;
    g.nbin = nb;
    g.inv_hb = (float)((double)nb / ext);
  }
  g.cap_mem = sphere_bound(g.w, sigma);
  g.cap_obj = sphere_bound(g.w + 2.0 * sigma, sigma);
  if ((int64_t)g.cap_mem > N) g.cap_mem = (int)N;
  if ((double)g.ncell * g.cap_mem > 2.0e9) {
    delete h;
    return fail3(ECMC_ERR_ARG, "too many cells");
  }
  int rc = layout3(h);
  if (rc) {
    delete h;
    return rc;
  }
  if (cudaStreamCreateWithFlags(&h->own, cudaStreamNonBlocking) != cudaSuccess) {
    delete h;
    return fail3(ECMC_ERR_CUDA, "stream creation failed");
  }
  h->stream = h->own;
  const size_t nn = (size_t)N;
  if (cudaMalloc(&h->px, sizeof(double) * nn) != cudaSuccess ||
      cudaMalloc(&h->py, sizeof(double) * nn) != cudaSuccess ||
      cudaMalloc(&h->pz, sizeof(double) * nn) != cudaSuccess ||
      cudaMalloc(&h->xyz_tmp, sizeof(double) * 3 * nn) != cudaSuccess ||
      cudaMalloc(&h->cnt, sizeof(int) * (size_t)g.ncell) != cudaSuccess ||
      cudaMalloc(&h->ids, sizeof(int) * (size_t)g.ncell * g.cap_mem) != cudaSuccess ||
      cudaMalloc(&h->cell_of, sizeof(int) * nn) != cudaSuccess ||
      cudaMalloc(&h->err, sizeof(int)) != cudaSuccess ||
      cudaMalloc(&h->cs, sizeof(Cell3) * (size_t)g.ncell) != cudaSuccess ||
      cudaMalloc(&h->st, sizeof(State3)) != cudaSuccess ||
      cudaMalloc(&h->tot, sizeof(Totals3)) != cudaSuccess ||
      cudaMalloc(&h->history, sizeof(double) * 2 * kHistoryCap) != cudaSuccess ||
      cudaMalloc(&h->hist_len, sizeof(int64_t)) != cudaSuccess ||
      cudaMalloc(&h->u64, sizeof(unsigned long long)) != cudaSuccess ||
      cudaMalloc(&h->sched, sizeof(unsigned) * 4) != cudaSuccess ||
      cudaMalloc(&h->done, sizeof(unsigned) * (size_t)g.ncell) != cudaSuccess) {
    cudaGetLastError();
    free3(h);
    delete h;
    return fail3(ECMC_ERR_OOM, "device allocation failed");
  }
  cudaMemsetAsync(h->sched, 0, sizeof(unsigned) * 4, h->stream);
  cudaMemsetAsync(h->done, 0, sizeof(unsigned) * (size_t)g.ncell, h->stream);
  // the cubic lattice start
  std::vector<double> xyz(3 * nn);
  const double a = L / (double)k;
  for (int64_t i = 0; i < N; ++i) {
    xyz[3 * i] = ((double)(i % k) + 0.5) * a;
    xyz[3 * i + 1] = ((double)((i / k) % k) + 0.5) * a;
    xyz[3 * i + 2] = ((double)(i / (k * k)) + 0.5) * a;
  }
  rc = ecmc3_set_positions(h, xyz.data(), 0, 0);
  if (rc) {
    free3(h);
    delete h;
    return rc;
  }
  *out = h;
  return ECMC_OK;
}

int ecmc3_destroy(ecmc3_t h) {
  if (!h) return ECMC_OK;  // like ecmc_destroy: nothing to release
  if (h->stream) cudaStreamSynchronize(h->stream);
  free3(h);
  delete h;
  return ECMC_OK;
}

int ecmc3_set_param(ecmc3_t h, int key, double v) {
  if (!h) return fail3(ECMC_ERR_ARG, "NULL handle");
  switch (key) {
    case ECMC3_PARAM_N_CHAINS: {
      const int n = (int)v;
      if ((double)n != v || n < 1 || n > (1 << 20)) return fail3(ECMC_ERR_ARG, "n_m");
      if (n != h->g.n_m) {
        h->g.n_m = n;
        cudaFree(h->recs);
        h->recs = nullptr;
      }
      return ECMC_OK;
    }
    case ECMC3_PARAM_REPLICA:
      if (!(v >= 0.0) || v != std::floor(v) || v > 9.0e15) return fail3(ECMC_ERR_ARG, "replica");
      h->g.replica = (uint64_t)v;
      return ECMC_OK;
    case ECMC3_PARAM_PERSISTENT:
      if (v != 0.0 && v != 1.0) return fail3(ECMC_ERR_ARG, "persistent must be 0 or 1");
      h->persistent = (int)v;
      return ECMC_OK;
    case ECMC3_PARAM_WAIT_LIMIT_MS:
      if (!(v >= 1.0 && v <= 600000.0)) return fail3(ECMC_ERR_ARG, "wait limit in [1, 600000] ms");
      h->wait_ns = (unsigned long long)(v * 1e6);
      return ECMC_OK;
    case ECMC3_PARAM_WAIT_TEST:
      if (v != 0.0 && v != 1.0) return fail3(ECMC_ERR_ARG, "wait test must be 0 or 1");
      h->wait_test = (int)v;
      return ECMC_OK;
    case ECMC3_PARAM_REPLAY:
      if (v != 0.0 && v != 1.0) return fail3(ECMC_ERR_ARG, "replay must be 0 or 1");
      h->g.replay = (int)v;
      return ECMC_OK;
    default:
      return fail3(ECMC_ERR_ARG, "unknown parameter %d", key);
  }
}

int ecmc3_get_param(ecmc3_t h, int key, double* v) {
  if (!h || !v) return fail3(ECMC_ERR_ARG, "NULL argument");
  switch (key) {
    case ECMC3_PARAM_N_CHAINS: *v = h->g.n_m; return ECMC_OK;
    case ECMC3_PARAM_REPLICA: *v = (double)h->g.replica; return ECMC_OK;
    case ECMC3_PARAM_PERSISTENT: *v = (h->persistent && h->fused_blocks > 0) ? 1.0 : 0.0;
      return ECMC_OK;
    case ECMC3_PARAM_WAIT_LIMIT_MS: *v = (double)h->wait_ns * 1e-6; return ECMC_OK;
    case ECMC3_PARAM_WAIT_TEST: *v = h->wait_test; return ECMC_OK;
    case ECMC3_PARAM_REPLAY: *v = h->g.replay; return ECMC_OK;
    default: return fail3(ECMC_ERR_ARG, "unknown parameter %d", key);
  }
}

int ecmc3_set_stream(ecmc3_t h, void* stream) {
  if (!h) return fail3(ECMC_ERR_ARG, "NULL handle");
  CK3(cudaStreamSynchronize(h->stream));
  h->stream = stream ? (cudaStream_t)stream : h->own;
  return ECMC_OK;
}

int ecmc3_set_positions(ecmc3_t h, const double* xyz, int on_device, int64_t t0) {
  if (!h || !xyz) return fail3(ECMC_ERR_ARG, "NULL argument");
  if (t0 < 0) return fail3(ECMC_ERR_ARG, "t0 must be >= 0");
  const double* src = xyz;
  if (!on_device) {
    CK3(cudaMemcpyAsync(h->xyz_tmp, xyz, sizeof(double) * 3 * (size_t)h->g.N,
                        cudaMemcpyHostToDevice, h->stream));
    src = h->xyz_tmp;
  }
  return load_dev(h, src, t0);
}

int ecmc3_positions(ecmc3_t h, double* xyz, int on_device) {
  if (!h || !xyz) return fail3(ECMC_ERR_ARG, "NULL argument");
  if (!h->valid) return fail3(ECMC_ERR_STATE, "state invalid after an earlier error");
  const Geom3& g = h->g;
  double* dst = on_device ? xyz : h->xyz_tmp;
  k3_join<<<(unsigned)((g.N + 255) / 256), 256, 0, h->stream>>>(h->px, h->py, h->pz, g.N, dst);
  CK3(cudaGetLastError());
  if (!on_device)
    CK3(cudaMemcpyAsync(xyz, h->xyz_tmp, sizeof(double) * 3 * (size_t)g.N,
                        cudaMemcpyDeviceToHost, h->stream));
  return check3(h);
}

int ecmc3_sweep(ecmc3_t h, int64_t n) {
  if (!h) return fail3(ECMC_ERR_ARG, "NULL handle");
  if (n < 0) return fail3(ECMC_ERR_ARG, "negative sweep count");
  if (!h->valid) return fail3(ECMC_ERR_STATE, "state invalid after an earlier error");
  const bool rec = n > 0;
  if (rec && !h->recs) {
    CK3(cudaMalloc(&h->recs, sizeof(int) * 4 * (size_t)h->g.ncell * h->g.n_m));
  }
  for (int64_t s = 0; s < n; ++s) {
    const int rc = enqueue_sweep(h, s == n - 1);
    if (rc) return rc;
  }
  h->t_host += n;
  return ECMC_OK;
}

int ecmc3_synchronize(ecmc3_t h) {
  if (!h) return fail3(ECMC_ERR_ARG, "NULL handle");
  return check3(h);
}

int ecmc3_sweep_index(ecmc3_t h, int64_t* t) {
  if (!h || !t) return fail3(ECMC_ERR_ARG, "NULL argument");
  *t = h->t_host;
  return ECMC_OK;
}

int ecmc3_counters(ecmc3_t h, ecmc_counters_t* out) {
  if (!h || !out) return fail3(ECMC_ERR_ARG, "NULL argument");
  Totals3 t;
  CK3(cudaMemcpyAsync(&t, h->tot, sizeof(t), cudaMemcpyDeviceToHost, h->stream));
  const int rc = check3(h);
  if (rc) return rc;
  std::memset(out, 0, sizeof(*out));
  out->sweeps = t.sweeps;
  out->chains = t.chains;
  out->events = t.events;
  out->lifts = t.lifts;
  out->frozen_hits = t.frozen;
  out->wall_hits = t.walls;
  out->replayed_legs = t.replayed;
  out->sum_b = t.sum_b;
  out->sum_disp = t.sum_disp;
  return ECMC_OK;
}

int ecmc3_pressure(ecmc3_t h, double* betaP, double* se) {
  if (!h || !betaP) return fail3(ECMC_ERR_ARG, "NULL argument");
  Totals3 t;
  int64_t n = 0;
  CK3(cudaMemcpyAsync(&t, h->tot, sizeof(t), cudaMemcpyDeviceToHost, h->stream));
  CK3(cudaMemcpyAsync(&n, h->hist_len, sizeof(n), cudaMemcpyDeviceToHost, h->stream));
  int rc = check3(h);
  if (rc) return rc;
  if (n < 1 || !(t.sum_disp_w > 0.0)) return fail3(ECMC_ERR_STATE, "no sweep since the last reset");
  const Geom3& g = h->g;
  const double rho_s3 = (double)g.N / (g.L * g.L * g.L) * g.sig2 * g.sigma;
  *betaP = rho_s3 * (1.0 + t.sum_b_w / t.sum_disp_w);
  if (se) {
    *se = 0.0;
    const int64_t m = n < kHistoryCap ? n : kHistoryCap;
    const int64_t nb = m >= 20 ? 20 : m;
    if (nb >= 2) {
      std::vector<double> hist(2 * (size_t)m);
      CK3(cudaMemcpyAsync(hist.data(), h->history, sizeof(double) * 2 * (size_t)m,
                          cudaMemcpyDeviceToHost, h->stream));
      CK3(cudaStreamSynchronize(h->stream));
      std::vector<double> vals;
      for (int64_t b = 0; b < nb; ++b) {
        const int64_t lo = b * m / nb, hi = (b + 1) * m / nb;
        double sb = 0.0, sd = 0.0;
        for (int64_t i = lo; i < hi; ++i) {
          sb += hist[2 * i];
          sd += hist[2 * i + 1];
        }
        vals.push_back(rho_s3 * (1.0 + sb / sd));
      }
      double mean = 0.0;
      for (double v : vals) mean += v;
      mean /= (double)nb;
      double var = 0.0;
      for (double v : vals) var += (v - mean) * (v - mean);
      *se = std::sqrt(var / (double)(nb - 1) / (double)nb);
    }
  }
  return ECMC_OK;
}

int ecmc3_reset_stats(ecmc3_t h) {
  if (!h) return fail3(ECMC_ERR_ARG, "NULL handle");
  CK3(cudaMemsetAsync(h->tot, 0, sizeof(Totals3), h->stream));
  CK3(cudaMemsetAsync(h->hist_len, 0, sizeof(int64_t), h->stream));
  return ECMC_OK;
}

int ecmc3_min_distance(ecmc3_t h, double* dmin) {
  if (!h || !dmin) return fail3(ECMC_ERR_ARG, "NULL argument");
  double d2 = 0.0;
  const int rc = min_dist2_3(h, &d2);
  if (rc) return rc;
  *dmin = std::sqrt(d2);
  return ECMC_OK;
}

int ecmc3_last_cells(ecmc3_t h, int32_t* cell_of_id) {
  if (!h || !cell_of_id) return fail3(ECMC_ERR_ARG, "NULL argument");
  CK3(cudaMemcpyAsync(cell_of_id, h->cell_of, sizeof(int32_t) * (size_t)h->g.N,
                      cudaMemcpyDeviceToHost, h->stream));
  return check3(h);
}

int ecmc3_chain_records(ecmc3_t h, int32_t* out) {
  if (!h || !out) return fail3(ECMC_ERR_ARG, "NULL argument");
  if (!h->recs) return fail3(ECMC_ERR_STATE, "no sweep has run");
  CK3(cudaMemcpyAsync(out, h->recs, sizeof(int32_t) * 4 * (size_t)h->g.ncell * h->g.n_m,
                      cudaMemcpyDeviceToHost, h->stream));
  return check3(h);
}

}  // extern "C"
