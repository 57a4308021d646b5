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
  int64_t t_host = 0;
  bool valid = false;
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
  for (int ci = 0; ci < 2; ++ci)
    ks_phase<<<(unsigned)(g.S / 2), kThreads, 0, h->stream>>>(
        g, h->st, ci, h->px, h->py, h->stripe_of, h->fU, h->fV, h->fkey, h->fid, h->fU0,
        h->stats, records ? h->recs : nullptr, h->err);
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
      cudaMalloc(&h->hist_len, sizeof(int64_t)) != cudaSuccess) {
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
