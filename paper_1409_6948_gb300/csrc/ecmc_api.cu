// ecmc_api.cu -- the C ABI of libecmc (declared in include/ecmc.h): handle
// life cycle, parameters, the sweep driver, and the data getters.
//
// One sweep (Sec. 3.4 steps 1-7) is the fixed launch sequence
//   draws -> binning -> 4 x (frame build, chain kernel) -> reduction,
// every kernel reading the sweep counter, shift and colour order from device
// memory; it is captured once into a CUDA graph per buffer parity and
// replayed.
#include <cmath>
#include <cstdarg>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "ecmc.h"
#include "ecmc_internal.cuh"

using namespace ecmc;

namespace {

thread_local char g_msg[512] = "";

int fail(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_msg, sizeof(g_msg), fmt, ap);
  va_end(ap);
  return code;
}

#define CK(call)                                                                          \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return fail(e_ == cudaErrorMemoryAllocation ? ECMC_ERR_OOM : ECMC_ERR_CUDA,         \
                  "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
  } while (0)

enum TimerClass { TC_BIN = 0, TC_FRAME = 1, TC_PHASE = 2, TC_OTHER = 3 };

}  // namespace

namespace ecmc {
int report_error(int code, const char* msg) { return fail(code, "%s", msg); }
}  // namespace ecmc

struct ecmc_ctx {
  std::vector<Geom> geo;        // host copy of every replica's geometry
  std::vector<int> cell_rep;    // replica of every global cell
  std::vector<int> act_rep;     // replica of every global active cell
  std::vector<int64_t> n_off;   // disk offsets, R + 1 entries
  Geom* d_geo = nullptr;
  int* d_cell_rep = nullptr;
  int* d_act_rep = nullptr;
  int64_t* d_n_off = nullptr;
  DevBufs b;
  RecLayout lay;
  int precision = 1;
  int tpc = 0;          // lanes per cell in use
  int tpc_param = 0;    // 0 = automatic
  int fmode = 0;        // frame placement in use (see phase_smem_bytes)
  int fmode_param = -1; // -1 = automatic
  int persist_param = 1; // 1 = one persistent launch per sweep when the frames fit
  int persistent = 0;    // in use
  int fused_blocks = 0;  // grid of the persistent sweep kernel
  double wait_ms = 5000.0;
  int n_sm = 0;
  std::vector<int2> chunks;
  std::vector<int> chunk_off;
  int2* d_chunks = nullptr;
  int* d_chunk_off = nullptr;
  ChunkSums* d_partials = nullptr;
  int warps = 0;
  int warps_param = 0;
  float strip_w = (float)kDefaultStripWidth;
  size_t records_cap = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t own_stream = nullptr;
  int64_t t_host = 0;          // mirror of the device sweep counter
  int64_t hist_len_host = 0;   // mirror of the history length
  bool valid_state = true;
  int record_chains = 0;
  int use_graph = 1;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  // timing
  int timing = 0;
  struct Ev {
    cudaEvent_t a, b;
    int cls;
  };
  std::vector<Ev> pending;
  std::vector<cudaEvent_t> pool;
  double ms[4] = {0, 0, 0, 0};
  int64_t launches[4] = {0, 0, 0, 0};
  // g(r): one histogram of gr_nbins bins per replica ([R][gr_nbins]) and
  // the number of measurements of each replica
  double gr_dr = 0.01, gr_rmax = 5.0;
  int gr_nbins = 0;
  unsigned long long* gr_counts = nullptr;
  std::vector<int64_t> gr_meas;
  // scratch
  double* xy_tmp = nullptr;
  int* int_tmp = nullptr;
  unsigned long long* u64_tmp = nullptr;
  UndoEntry* undo = nullptr;  // rejecting boundary rule: [C_total][cap] undo logs
  // pinned staging for the small copies of ecmc_set_positions, so that the
  // whole load (states up, binning, overlap check, result down) needs one
  // synchronisation
  SweepState* pin_states = nullptr;       // [R]
  unsigned long long* pin_bits = nullptr;  // [2]: initial and resulting minimum
};

namespace {

int compute_layout(ecmc_ctx* h);

double packing_bound(double W, double H, double sigma) {
  // disjoint disks of diameter sigma' = sigma (1 - 1e-6) whose centres lie in
  // a W x H rectangle fit, with their full area, in the rectangle grown by
  // sigma'/2 on every side
  const double sp = sigma * (1.0 - 1e-6);
  const double pi = 3.14159265358979323846;
  return (W + sp) * (H + sp) / (pi * sp * sp / 4.0);
}

}  // namespace

namespace ecmc {

void set_screen_bounds(Geom& g) {
  // M: power of two bounding every frame coordinate, |v| < max(w,h) + sigma
  const double ext = (g.w > g.h ? g.w : g.h) + 1.01 * g.sigma;
  double M = 1.0;
  while (M < ext) M *= 2.0;
  // |FP32 difference - FP64 difference| <= 6 * 2^-24 * M + tiny: each FP32
  // operand is within 2^-23 M of its FP64 value (rounded to nearest in the
  // frame builder, truncated toward zero after a move), the FP32 difference
  // adds 2^-23 M, the FP64 difference 2^-52 M
  const double e = 6.5 * std::ldexp(1.0, -24) * M;
  const double sig = g.sigma;
  // |x32 - (sigma^2 - ddy^2)| <= ex, x32 = fma(-|db|, |db|, sigma^2) in FP32
  const double ex = (2.0 * sig + 2.0 * e) * e + 3.0 * std::ldexp(1.0, -24) * sig * sig;
  // hit distance: e (along d) + sqrt(ex) (sqrt is 1/2-Hoelder) + rsqrt
  // approximation + FP32 rounding of the difference, with 25% slack
  const double sm = 1.25 * (e + std::sqrt(ex) + std::ldexp(1.0, -20) * sig +
                            std::ldexp(1.0, -23) * (2.0 * M + sig));
  g.eps_d = (float)(e * 1.0000001);
  g.s_margin = (float)sm;
  g.sig_plus = std::nextafter((float)(sig + e + std::ldexp(sig, -40)), 1e30f);
  g.sig_minus = std::nextafter((float)(sig - e - std::ldexp(sig, -40)), -1e30f);
  g.sig2f = (float)(sig * sig);
  g.sigf = (float)sig;
  // isotropic chains: the FP32 frame differences are within 1.5 * 2^-22 M of
  // the FP64 ones; the FP32 projections on a unit direction rounded to FP32
  // (two products and a sum) within 6 * 2^-22 M; twice that as the bound
  g.iso_e = (float)(12.0 * std::ldexp(1.0, -22) * M + std::ldexp(sig, -40));
  // sqrt(sigma^2 - c^2) from FP32 operands: |x32 - x| <= 3 * 2^-24 sigma^2, and
  // the square root is 1/2-Hoelder: sqrt(3 * 2^-24) sigma < 2^-11 sigma
  g.iso_sq = (float)(std::ldexp(sig, -11) + std::ldexp(sig, -22));
  g.iso_r = (float)(std::ldexp(1.0, -22) * (2.0 * M + sig));
  g.iso_sig_lo = std::nextafter((float)(sig * (1.0 - std::ldexp(1.0, -21))), -1e30f);
  g.iso_sig_hi = std::nextafter((float)(sig * (1.0 + std::ldexp(1.0, -21))), 1e30f);
  g.strip_margin = (float)(4.0 * e + 1e-5 * sig);
}

void set_strip_bins(Geom& g, double strip_w) {
  const double bw = strip_w * g.sigma;
  const double extB = (g.w > g.h ? g.w : g.h) + 2.0 * g.sigma;
  g.nbin = (int)std::ceil(extB / bw) + 1;
  g.bin_w = (float)bw;
  g.inv_bin_w = (float)(1.0 / bw);
}

}  // namespace ecmc

namespace {

int upload_geometry(ecmc_ctx* h) {
  CK(cudaMemcpyAsync(h->d_geo, h->geo.data(), sizeof(Geom) * h->geo.size(),
                     cudaMemcpyHostToDevice, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return ECMC_OK;
}

RecLayout layout_for(ecmc_ctx* h, int tpc) {
  int nbin = 0, cap_obj = 0;
  for (const Geom& g : h->geo) {
    nbin = g.nbin > nbin ? g.nbin : nbin;
    cap_obj = g.cap_obj > cap_obj ? g.cap_obj : cap_obj;
  }
  return make_layout(32 / tpc, nbin, h->b.cap, cap_obj);
}

int choose_tpc(ecmc_ctx* h, int fmode) {
  if (h->tpc_param) return h->tpc_param;
  // the widest group (most cells per warp) whose frames leave room for at
  // least four warps per SM, but at most 8 cells per warp: measured on GB300
  // at N = 1M, eta = 0.72, 8 cells per warp beat 4, 16 and 32
  for (int t = 4; t <= 32; t *= 2)
    if (phase_smem_bytes(layout_for(h, t), 1, fmode) <= 52 * 1024) return t;
  return 32;
}

int compute_layout(ecmc_ctx* h) {
  for (Geom& g : h->geo) set_strip_bins(g, h->strip_w);
  const size_t limit = 232448;  // opt-in shared memory per block on sm_103
  if (h->n_sm == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&h->n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (h->n_sm <= 0) h->n_sm = 1;
  }
  // frame placement: whole frames in shared memory when every group of the
  // phase fits at once, else only the light part (FP64 in global memory);
  // frames too large for shared memory are used in place in global memory
  int fmode = h->fmode_param;
  if (fmode < 0) {
    const int t0 = choose_tpc(h, 0);
    const RecLayout l0 = layout_for(h, t0);
    const size_t groups = (size_t)(h->b.A_total + l0.cpw - 1) / l0.cpw;
    const size_t total = groups * phase_smem_bytes(l0, 1, 0);
    fmode = (phase_smem_bytes(l0, 1, 0) <= limit &&
             total <= (size_t)h->n_sm * limit * 9 / 10) ? 0 : 1;
  }
  h->tpc = choose_tpc(h, fmode);
  h->lay = layout_for(h, h->tpc);
  if (fmode < 2 && phase_smem_bytes(h->lay, 1, fmode) > limit) {
    if (h->tpc_param && h->tpc_param != 32)
      return fail(ECMC_ERR_UNSUPPORTED, "cell frames too large for %d lanes per cell",
                  h->tpc_param);
    h->tpc = 32;
    h->lay = layout_for(h, 32);
    if (phase_smem_bytes(h->lay, 1, fmode) > limit) fmode = 1;
    if (phase_smem_bytes(h->lay, 1, fmode) > limit) fmode = 2;
  }
  h->fmode = fmode;
  h->b.fmode = fmode;
  const size_t per_warp = phase_smem_bytes(h->lay, 1, fmode);
  int w = h->warps_param;
  if (w == 0) w = 1;  // one warp per block spreads the groups over every SM
  if (per_warp > 0 && (size_t)w * per_warp > limit) w = (int)(limit / per_warp);
  if (w < 1) w = 1;
  h->warps = w;
  const int n_groups = (h->b.A_total + h->lay.cpw - 1) / h->lay.cpw;
  const size_t need = (size_t)n_groups * h->lay.bytes;
  if (need > h->records_cap) {
    if (h->b.records) cudaFree(h->b.records);
    h->b.records = nullptr;
    CK(cudaMalloc(&h->b.records, need));
    h->records_cap = need;
  }
  if (h->b.gtouch) cudaFree(h->b.gtouch);
  h->b.gtouch = nullptr;
  if (fmode == 2)
    CK(cudaMalloc(&h->b.gtouch, (size_t)n_groups * align16((size_t)h->lay.cap_obj * h->lay.cpw)));
  if (h->b.stage) cudaFree(h->b.stage);
  h->b.stage = nullptr;
  h->b.stage_bytes = 0;
  if (frame_build_smem(h->lay) > limit) {
    h->b.stage_bytes = frame_stage_bytes(h->lay);
    CK(cudaMalloc(&h->b.stage, h->b.stage_bytes * (size_t)h->b.A_total));
  }
  if ((!h->b.stage && configure_frame_build(h->lay)) ||
      configure_phase(h->lay, h->tpc, h->warps, fmode))
    return fail(ECMC_ERR_CUDA, "kernel configuration failed: %s",
                cudaGetErrorString(cudaGetLastError()));
  // one persistent launch per sweep when a warp's frames, histories and
  // builder scratch fit in shared memory at least twice per SM
  h->persistent = 0;
  h->fused_blocks = 0;
  // the persistent kernel keeps its frames in shared memory (frame mode 0)
  // unless mode 1 is asked for: FP64 coordinates in a per-warp scratch area of
  // global memory, more warps per SM (measured at N = 1M, eta = 0.72: 1.64
  // against 1.58 * 10^9 events/s); isotropic chains use mode 0
  const int fm = (h->fmode_param == 1 && chain_kind(h->b) == 0) ? 1 : 0;
  if (h->persist_param && fmode < 2 && fused_smem_bytes(h->lay, fm) <= limit / 2) {
    int per_sm = 0;
    if (configure_fused(h->lay, h->tpc, fm, chain_kind(h->b), &per_sm) == 0) {
      const int n_items = 4 * n_groups;
      const int grid = per_sm * h->n_sm < n_items ? per_sm * h->n_sm : n_items;
      const size_t scratch = (size_t)grid * fused_scratch_bytes(h->lay);
      if (scratch > h->records_cap) {
        cudaFree(h->b.records);
        h->b.records = nullptr;
        CK(cudaMalloc(&h->b.records, scratch));
        h->records_cap = scratch;
      }
      h->fused_blocks = grid;
      h->persistent = 1;
      h->fmode = fm;
      h->b.fmode = fm;
    } else {
      cudaGetLastError();
    }
  }
  return upload_geometry(h);
}

void drop_graphs(ecmc_ctx* h) {
  for (int i = 0; i < 2; ++i)
    if (h->graph[i]) {
      cudaGraphExecDestroy(h->graph[i]);
      h->graph[i] = nullptr;
    }
}

cudaEvent_t get_event(ecmc_ctx* h) {
  if (!h->pool.empty()) {
    cudaEvent_t e = h->pool.back();
    h->pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  cudaEventCreate(&e);
  return e;
}

struct Timed {
  ecmc_ctx* h;
  int cls;
  cudaEvent_t a = nullptr;
  Timed(ecmc_ctx* hh, int c) : h(hh), cls(c) {
    if (h->timing) {
      a = get_event(h);
      cudaEventRecord(a, h->stream);
    }
  }
  ~Timed() {
    if (h->timing) {
      cudaEvent_t b = get_event(h);
      cudaEventRecord(b, h->stream);
      h->pending.push_back({a, b, cls});
    }
    h->launches[cls] += 1;
  }
};

void harvest_timing(ecmc_ctx* h) {
  for (auto& e : h->pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, e.a, e.b) == cudaSuccess) h->ms[e.cls] += ms;
    h->pool.push_back(e.a);
    h->pool.push_back(e.b);
  }
  h->pending.clear();
}

// Enqueue one sweep of every replica (no graph).
int enqueue_sweep(ecmc_ctx* h) {
  const int src = h->b.cur, dst = 1 - h->b.cur;
  if (h->record_chains && h->b.chain_recs)
    CK(cudaMemsetAsync(h->b.chain_recs, 0xff,
                       sizeof(ChainRec) * (size_t)h->b.C_total * h->b.rec_stride, h->stream));
  {
    Timed tm(h, TC_BIN);
    launch_sweep_begin(h->b, h->stream);
    launch_bin(h->b, src, dst, h->stream);
  }
  h->b.cur = dst;
  if (h->persistent) {
    {
      Timed tm(h, TC_PHASE);
      if (launch_fused(h->b, h->lay, h->tpc, h->fused_blocks, h->record_chains, h->precision,
                       h->stream))
        return fail(ECMC_ERR_CUDA, "sweep kernel launch failed: %s",
                    cudaGetErrorString(cudaGetLastError()));
    }
    {
      Timed tm(h, TC_OTHER);
      launch_sweep_end(h->b, h->stream);
    }
    CK(cudaGetLastError());
    return ECMC_OK;
  }
  for (int ci = 0; ci < 4; ++ci) {
    {
      Timed tm(h, TC_FRAME);
      launch_frame_build(h->b, h->lay, ci, h->stream);
    }
    {
      Timed tm(h, TC_PHASE);
      if (launch_phase(h->b, h->lay, ci, h->tpc, h->warps, h->record_chains, h->precision,
                       h->stream))
        return fail(ECMC_ERR_CUDA, "chain kernel launch failed: %s",
                    cudaGetErrorString(cudaGetLastError()));
    }
  }
  {
    Timed tm(h, TC_OTHER);
    launch_sweep_end(h->b, h->stream);
  }
  CK(cudaGetLastError());
  return ECMC_OK;
}

int ensure_history(ecmc_ctx* h, int64_t extra) {
  const int64_t need = h->hist_len_host + extra;
  if (need <= h->b.history_cap) return ECMC_OK;
  int64_t cap = h->b.history_cap ? h->b.history_cap : 1024;
  while (cap < need) cap *= 2;
  double* nh = nullptr;
  CK(cudaMalloc(&nh, sizeof(double) * 2 * (size_t)cap * h->b.R));
  if (h->b.history && h->hist_len_host > 0) {
    const int64_t len = h->hist_len_host < h->b.history_cap ? h->hist_len_host : h->b.history_cap;
    CK(cudaMemcpy2DAsync(nh, sizeof(double) * 2 * cap, h->b.history,
                         sizeof(double) * 2 * h->b.history_cap, sizeof(double) * 2 * len, h->b.R,
                         cudaMemcpyDeviceToDevice, h->stream));
  }
  CK(cudaStreamSynchronize(h->stream));
  if (h->b.history) cudaFree(h->b.history);
  h->b.history = nh;
  h->b.history_cap = cap;
  drop_graphs(h);  // the graphs hold the old pointer
  return ECMC_OK;
}

int check_device_error(ecmc_ctx* h) {
  int e = 0;
  CK(cudaMemcpyAsync(&e, h->b.err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (h->timing) harvest_timing(h);
  if (e == DEV_CAPACITY) {
    h->valid_state = false;
    return fail(ECMC_ERR_CAPACITY, "a cell bucket or frame exceeded its packing bound");
  }
  if (e == DEV_CHAIN_CAP) {
    h->valid_state = false;
    return fail(ECMC_ERR_CHAIN_CAP, "a chain reached the per-chain event cap");
  }
  if (e == DEV_WAIT_TIMEOUT) {
    h->valid_state = false;
    CK(cudaMemsetAsync(h->b.err, 0, sizeof(int), h->stream));
    return fail(ECMC_ERR_TIMEOUT,
                "a dependency wait of the persistent sweep kernel exceeded %.0f ms; the sweep "
                "was abandoned (positions must be set again)", h->wait_ms);
  }
  return ECMC_OK;
}

// smallest pair distance squared over all replicas (pairs closer than 2
// sigma), enqueued: the result lands in pin_bits[1] once the stream has
// passed it
int enqueue_min_dist2(ecmc_ctx* h) {
  double sig_max = 0.0;
  for (const Geom& g : h->geo) sig_max = g.sigma > sig_max ? g.sigma : sig_max;
  const double r2 = 4.0 * sig_max * sig_max;
  std::memcpy(&h->pin_bits[0], &r2, sizeof(r2));
  CK(cudaMemcpyAsync(h->u64_tmp, &h->pin_bits[0], sizeof(unsigned long long),
                     cudaMemcpyHostToDevice, h->stream));
  for (const Geom& g : h->geo) launch_min_dist(g, h->b, 2.0 * g.sigma, h->u64_tmp, h->stream);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(&h->pin_bits[1], h->u64_tmp, sizeof(unsigned long long),
                     cudaMemcpyDeviceToHost, h->stream));
  return ECMC_OK;
}

int min_dist2(ecmc_ctx* h, double* d2) {
  int rc = enqueue_min_dist2(h);
  if (rc) return rc;
  rc = check_device_error(h);
  if (rc) return rc;
  std::memcpy(d2, &h->pin_bits[1], sizeof(*d2));
  return ECMC_OK;
}

int load_positions_dev(ecmc_ctx* h, const double* xy_dev, int64_t t0) {
  launch_load_flat(h->b, xy_dev, h->stream);
  for (int r = 0; r < h->b.R; ++r) {
    SweepState& v = h->pin_states[r];
    std::memset(&v, 0, sizeof(v));
    v.t = t0;
    v.history_len = h->hist_len_host;
  }
  CK(cudaMemcpyAsync(h->b.state, h->pin_states, sizeof(SweepState) * (size_t)h->b.R,
                     cudaMemcpyHostToDevice, h->stream));
  launch_sweep_begin(h->b, h->stream);
  launch_bin(h->b, -1, h->b.cur, h->stream);
  CK(cudaGetLastError());
  h->t_host = t0;
  h->valid_state = true;
  // the overlap check follows in the same stream; one synchronisation reports
  // a binning error and delivers the smallest distance
  int rc = enqueue_min_dist2(h);
  if (rc) return rc;
  rc = check_device_error(h);
  if (rc) return rc;
  double d2 = 0.0;
  std::memcpy(&d2, &h->pin_bits[1], sizeof(d2));
  // no two disks may overlap beyond rounding
  double sig2_min = 1e300;
  for (const Geom& g : h->geo) sig2_min = g.sig2 < sig2_min ? g.sig2 : sig2_min;
  if (d2 < sig2_min * (1.0 - 1e-9)) {
    h->valid_state = false;
    return fail(ECMC_ERR_OVERLAP, "positions overlap: smallest distance %.17g < sigma",
                std::sqrt(d2));
  }
  return ECMC_OK;
}

int default_nm(const Geom& g) {
  const double pi = 3.14159265358979323846;
  const double eta = (double)g.N * pi * g.sigma * g.sigma / (4.0 * g.L * g.L);
  const double eta_hcp = pi / (2.0 * std::sqrt(3.0));
  const double lambda0 = g.sigma * (eta_hcp - eta) / (2.0 * eta_hcp);
  if (!(g.ell > 0.0) || !(lambda0 > 0.0)) return 1;
  const double nm = (double)g.N / (double)g.ncell * lambda0 / g.ell;
  const double r = std::floor(nm + 0.5);
  if (r < 1.0) return 1;
  if (r > 1e6) return 1000000;
  return (int)r;
}

int realloc_chain_recs(ecmc_ctx* h) {
  if (h->b.chain_recs) cudaFree(h->b.chain_recs);
  h->b.chain_recs = nullptr;
  int stride = 1;
  for (const Geom& g : h->geo) stride = g.n_m > stride ? g.n_m : stride;
  h->b.rec_stride = stride;
  if (!h->record_chains) return ECMC_OK;
  const size_t n = (size_t)h->b.C_total * stride;
  CK(cudaMalloc(&h->b.chain_recs, sizeof(ChainRec) * n));
  CK(cudaMemsetAsync(h->b.chain_recs, 0xff, sizeof(ChainRec) * n, h->stream));
  return ECMC_OK;
}

void free_all(ecmc_ctx* h) {
  drop_graphs(h);
  for (int i = 0; i < 2; ++i) {
    cudaFree(h->b.px[i]);
    cudaFree(h->b.py[i]);
    cudaFree(h->b.pid[i]);
    cudaFree(h->b.count[i]);
  }
  cudaFree(h->b.state);
  cudaFree(h->b.cell_stats);
  cudaFree(h->b.totals);
  cudaFree(h->b.history);
  cudaFree(h->b.records);
  cudaFree(h->b.gtouch);
  cudaFree(h->b.stage);
  cudaFree(h->b.err);
  cudaFree(h->b.sched);
  cudaFree(h->b.done);
  cudaFree(h->b.chain_recs);
  cudaFree(h->d_geo);
  cudaFree(h->d_cell_rep);
  cudaFree(h->d_act_rep);
  cudaFree(h->d_n_off);
  cudaFree(h->d_chunks);
  cudaFree(h->d_chunk_off);
  cudaFree(h->d_partials);
  cudaFree(h->gr_counts);
  cudaFree(h->xy_tmp);
  cudaFree(h->int_tmp);
  cudaFree(h->u64_tmp);
  cudaFree(h->undo);
  cudaFreeHost(h->pin_states);
  cudaFreeHost(h->pin_bits);
  for (auto& e : h->pending) {
    cudaEventDestroy(e.a);
    cudaEventDestroy(e.b);
  }
  for (auto e : h->pool) cudaEventDestroy(e);
  if (h->own_stream) cudaStreamDestroy(h->own_stream);
}

int setup_gr(ecmc_ctx* h) {
  const Geom& g = h->geo[0];
  const int nb = (int)std::floor((h->gr_rmax - g.sigma) / h->gr_dr + 0.5);
  if (nb < 1 || nb > 1000000) return fail(ECMC_ERR_ARG, "bad g(r) binning");
  if (h->gr_counts) cudaFree(h->gr_counts);
  h->gr_counts = nullptr;
  h->gr_nbins = nb;
  const size_t total = (size_t)nb * h->geo.size();
  CK(cudaMalloc(&h->gr_counts, sizeof(unsigned long long) * total));
  CK(cudaMemsetAsync(h->gr_counts, 0, sizeof(unsigned long long) * total, h->stream));
  h->gr_meas.assign(h->geo.size(), 0);
  return ECMC_OK;
}

// Geometry, capacities and FP32 screening bounds of one replica.  With
// lattice_start, N must be a perfect square whose lattice does not overlap.
int setup_geom(const ecmc_replica_desc_t& d, Geom& g, bool lattice_start = true) {
  const int64_t N = d.N;
  if (N < 1 || N >= (int64_t(1) << 27)) return fail(ECMC_ERR_ARG, "N out of range");
  const int64_t k = (int64_t)std::llround(std::sqrt((double)N));
  if (lattice_start && k * k != N)
    return fail(ECMC_ERR_ARG, "N must be a perfect square (lattice start)");
  if (!(d.L > 0.0) || !(d.sigma > 0.0) || !std::isfinite(d.L) || !std::isfinite(d.sigma))
    return fail(ECMC_ERR_ARG, "L and sigma must be positive");
  // sigma^2 - c^2 and every frame coordinate stay normal numbers in FP64 and FP32
  if (!(d.sigma >= std::ldexp(1.0, -40) && d.sigma <= std::ldexp(1.0, 40)) ||
      !(d.L < std::ldexp(d.sigma, 40)))
    return fail(ECMC_ERR_ARG, "sigma must lie in [2^-40, 2^40] and L below 2^40 sigma");
  if (d.cells_x < 2 || d.cells_y < 2 || (d.cells_x & 1) || (d.cells_y & 1))
    return fail(ECMC_ERR_ARG, "cells per side must be even and >= 2");
  if (!(d.L / d.cells_x > d.sigma) || !(d.L / d.cells_y > d.sigma))
    return fail(ECMC_ERR_ARG, "cell side must exceed sigma");
  if (lattice_start && !(d.L / (double)k > d.sigma))
    return fail(ECMC_ERR_ARG, "square lattice would overlap");
  if (!(d.ell >= 0.0) || !std::isfinite(d.ell)) return fail(ECMC_ERR_ARG, "ell must be >= 0");
  if ((int64_t)d.cells_x * d.cells_y > (int64_t(1) << 26))
    return fail(ECMC_ERR_ARG, "too many cells");
  if (d.n_m < 0 || d.n_m > 1000000) return fail(ECMC_ERR_ARG, "n_m out of range");
  std::memset(&g, 0, sizeof(g));
  g.N = N;
  g.L = d.L;
  g.sigma = d.sigma;
  g.sig2 = d.sigma * d.sigma;
  g.cells_x = d.cells_x;
  g.cells_y = d.cells_y;
  g.ncell = d.cells_x * d.cells_y;
  g.nact = (d.cells_x / 2) * (d.cells_y / 2);
  g.w = d.L / (double)d.cells_x;
  g.h = d.L / (double)d.cells_y;
  g.inv_w = 1.0 / g.w;
  g.inv_h = 1.0 / g.h;
  set_bin_screen(g);
  g.ell = d.ell;
  g.seed = d.seed;
  g.replica = d.replica;
  g.dir_mode = 0;
  g.precision = 1;
  g.cap_mem = (int)std::floor(packing_bound(g.w, g.h, d.sigma)) + 2;
  g.cap_obj = (int)std::floor(packing_bound(g.w + 2 * d.sigma, g.h + 2 * d.sigma, d.sigma)) + 2;
  if (g.cap_mem > g.cap_obj) g.cap_mem = g.cap_obj;
  if ((int64_t)g.ncell * g.cap_mem < N)
    return fail(ECMC_ERR_ARG, "N exceeds the packing capacity of the box");
  g.n_m = d.n_m ? d.n_m : default_nm(g);
  set_screen_bounds(g);
  return ECMC_OK;
}

}  // namespace

namespace ecmc {
int setup_replica_geom(const ecmc_replica_desc_t& d, Geom& g, int lattice_start) {
  return setup_geom(d, g, lattice_start != 0);
}
}  // namespace ecmc

namespace {

int create_impl(ecmc_t* out, const ecmc_replica_desc_t* desc, int R) {
  if (!out) return fail(ECMC_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!desc || R < 1) return fail(ECMC_ERR_ARG, "need at least one replica");
  ecmc_ctx* h = new (std::nothrow) ecmc_ctx();
  if (!h) return fail(ECMC_ERR_OOM, "host allocation failed");
  std::memset(&h->b, 0, sizeof(h->b));
  h->b.replay = 1;
  auto bail = [&](int rc) {
    free_all(h);
    delete h;
    return rc;
  };
  h->geo.resize(R);
  h->n_off.assign(R + 1, 0);
  int64_t C_total = 0, A_total = 0;
  int cap = 0;
  for (int r = 0; r < R; ++r) {
    int rc = setup_geom(desc[r], h->geo[r]);
    if (rc) {
      delete h;
      return rc;
    }
    Geom& g = h->geo[r];
    g.rep = r;
    g.n_off = h->n_off[r];
    g.cell_off = (int)C_total;
    g.act_off = (int)A_total;
    h->n_off[r + 1] = h->n_off[r] + g.N;
    C_total += g.ncell;
    A_total += g.nact;
    cap = g.cap_mem > cap ? g.cap_mem : cap;
    if (C_total >= (int64_t(1) << 30)) {
      delete h;
      return fail(ECMC_ERR_ARG, "too many cells in the batch");
    }
  }
  for (int r = 0; r < R; ++r) {
    h->cell_rep.insert(h->cell_rep.end(), h->geo[r].ncell, r);
    h->act_rep.insert(h->act_rep.end(), h->geo[r].nact, r);
  }
  // end-of-sweep reduction chunks: at most 2048 cells, never across replicas
  h->chunk_off.assign(1, 0);
  for (int r = 0; r < R; ++r) {
    const Geom& g = h->geo[r];
    for (int c0 = 0; c0 < g.ncell; c0 += 2048) {
      const int c1 = c0 + 2048 < g.ncell ? c0 + 2048 : g.ncell;
      h->chunks.push_back(make_int2(g.cell_off + c0, g.cell_off + c1));
    }
    h->chunk_off.push_back((int)h->chunks.size());
  }
  const int64_t N_total = h->n_off[R];
  if (N_total >= (int64_t(1) << 31) || C_total * (int64_t)cap >= (int64_t(1) << 31)) {
    delete h;
    return fail(ECMC_ERR_ARG, "batch too large");
  }
  DevBufs& b = h->b;
  b.R = R;
  b.C_total = (int)C_total;
  b.A_total = (int)A_total;
  b.cap = cap;
  b.N_total = N_total;
  b.cur = 0;

  if (cudaStreamCreateWithFlags(&h->own_stream, cudaStreamNonBlocking) != cudaSuccess)
    return bail(fail(ECMC_ERR_CUDA, "cannot create a stream (no CUDA device?)"));
  h->stream = h->own_stream;
  const size_t slots = (size_t)C_total * cap;
  for (int i = 0; i < 2; ++i) {
    if (cudaMalloc(&b.px[i], sizeof(double) * slots) != cudaSuccess ||
        cudaMalloc(&b.py[i], sizeof(double) * slots) != cudaSuccess ||
        cudaMalloc(&b.pid[i], sizeof(int) * slots) != cudaSuccess ||
        cudaMalloc(&b.count[i], sizeof(int) * (size_t)C_total) != cudaSuccess)
      return bail(fail(ECMC_ERR_OOM, "device allocation of %zu slots failed", slots));
    cudaMemsetAsync(b.count[i], 0, sizeof(int) * (size_t)C_total, h->stream);
  }
  if (cudaMalloc(&b.state, sizeof(SweepState) * R) != cudaSuccess ||
      cudaMalloc(&b.cell_stats, sizeof(CellStats) * (size_t)C_total) != cudaSuccess ||
      cudaMalloc(&b.totals, sizeof(RunTotals) * R) != cudaSuccess ||
      cudaMalloc(&b.err, sizeof(int)) != cudaSuccess ||
      cudaMalloc(&b.sched, sizeof(unsigned) * 4) != cudaSuccess ||
      cudaMalloc(&b.done, sizeof(unsigned) * (size_t)C_total) != cudaSuccess ||
      cudaMalloc(&h->d_geo, sizeof(Geom) * R) != cudaSuccess ||
      cudaMalloc(&h->d_cell_rep, sizeof(int) * (size_t)C_total) != cudaSuccess ||
      cudaMalloc(&h->d_act_rep, sizeof(int) * (size_t)A_total) != cudaSuccess ||
      cudaMalloc(&h->d_n_off, sizeof(int64_t) * (R + 1)) != cudaSuccess ||
      cudaMalloc(&h->d_chunks, sizeof(int2) * h->chunks.size()) != cudaSuccess ||
      cudaMalloc(&h->d_chunk_off, sizeof(int) * h->chunk_off.size()) != cudaSuccess ||
      cudaMalloc(&h->d_partials, sizeof(ChunkSums) * h->chunks.size()) != cudaSuccess ||
      cudaMalloc(&h->xy_tmp, sizeof(double) * 2 * (size_t)N_total) != cudaSuccess ||
      cudaMalloc(&h->int_tmp, sizeof(int) * (size_t)N_total) != cudaSuccess ||
      cudaMalloc(&h->u64_tmp, sizeof(unsigned long long) * 4) != cudaSuccess ||
      cudaMallocHost(&h->pin_states, sizeof(SweepState) * R) != cudaSuccess ||
      cudaMallocHost(&h->pin_bits, sizeof(unsigned long long) * 2) != cudaSuccess)
    return bail(fail(ECMC_ERR_OOM, "device allocation failed"));
  cudaMemsetAsync(b.totals, 0, sizeof(RunTotals) * R, h->stream);
  cudaMemsetAsync(b.err, 0, sizeof(int), h->stream);
  cudaMemsetAsync(b.sched, 0, sizeof(unsigned) * 4, h->stream);
  cudaMemsetAsync(b.done, 0, sizeof(unsigned) * (size_t)C_total, h->stream);
  b.wait_ns = (unsigned long long)(h->wait_ms * 1e6);
  cudaMemsetAsync(b.cell_stats, 0, sizeof(CellStats) * (size_t)C_total, h->stream);
  if (cudaMemcpyAsync(h->d_cell_rep, h->cell_rep.data(), sizeof(int) * C_total,
                      cudaMemcpyHostToDevice, h->stream) != cudaSuccess ||
      cudaMemcpyAsync(h->d_act_rep, h->act_rep.data(), sizeof(int) * A_total,
                      cudaMemcpyHostToDevice, h->stream) != cudaSuccess ||
      cudaMemcpyAsync(h->d_n_off, h->n_off.data(), sizeof(int64_t) * (R + 1),
                      cudaMemcpyHostToDevice, h->stream) != cudaSuccess ||
      cudaMemcpyAsync(h->d_chunks, h->chunks.data(), sizeof(int2) * h->chunks.size(),
                      cudaMemcpyHostToDevice, h->stream) != cudaSuccess ||
      cudaMemcpyAsync(h->d_chunk_off, h->chunk_off.data(), sizeof(int) * h->chunk_off.size(),
                      cudaMemcpyHostToDevice, h->stream) != cudaSuccess)
    return bail(fail(ECMC_ERR_CUDA, "upload failed"));
  b.chunks = h->d_chunks;
  b.chunk_off = h->d_chunk_off;
  b.partials = h->d_partials;
  b.n_chunks = (int)h->chunks.size();
  b.rg = h->d_geo;
  b.cell_rep = h->d_cell_rep;
  b.act_rep = h->d_act_rep;
  b.n_off = h->d_n_off;
  int rc = compute_layout(h);
  if (rc) return bail(rc);
  rc = realloc_chain_recs(h);
  if (rc) return bail(rc);
  rc = ensure_history(h, 1024);
  if (rc) return bail(rc);
  rc = setup_gr(h);
  if (rc) return bail(rc);

  // square-lattice start of every replica
  std::vector<double> xy(2 * (size_t)N_total);
  for (int r = 0; r < R; ++r) {
    const Geom& g = h->geo[r];
    const int64_t k = (int64_t)std::llround(std::sqrt((double)g.N));
    const double a = g.L / (double)k;
    double* p = xy.data() + 2 * g.n_off;
    for (int64_t i = 0; i < g.N; ++i) {
      p[2 * i] = ((double)(i % k) + 0.5) * a;
      p[2 * i + 1] = ((double)(i / k) + 0.5) * a;
    }
  }
  if (cudaMemcpyAsync(h->xy_tmp, xy.data(), sizeof(double) * xy.size(), cudaMemcpyHostToDevice,
                      h->stream) != cudaSuccess)
    return bail(fail(ECMC_ERR_CUDA, "upload failed"));
  rc = load_positions_dev(h, h->xy_tmp, 0);
  if (rc) return bail(rc);
  *out = h;
  return ECMC_OK;
}

int pressure_of(ecmc_ctx* h, int r, double* betaP, double* se) {
  const int64_t n = h->hist_len_host < h->b.history_cap ? h->hist_len_host : h->b.history_cap;
  if (n < 1) return fail(ECMC_ERR_STATE, "no sweep since the last reset");
  const Geom& g = h->geo[r];
  std::vector<double> hist(2 * (size_t)n);
  CK(cudaMemcpyAsync(hist.data(), h->b.history + 2 * (size_t)r * h->b.history_cap,
                     sizeof(double) * 2 * n, cudaMemcpyDeviceToHost, h->stream));
  RunTotals t;
  CK(cudaMemcpyAsync(&t, h->b.totals + r, sizeof(t), cudaMemcpyDeviceToHost, h->stream));
  int rc = check_device_error(h);
  if (rc) return rc;
  const double rho_s2 = (double)g.N / (g.L * g.L) * g.sig2;
  if (!(t.sum_disp_w > 0.0)) return fail(ECMC_ERR_STATE, "no displacement since the last reset");
  *betaP = rho_s2 * (1.0 + t.sum_b_w / t.sum_disp_w);
  if (se) {
    *se = 0.0;
    const int64_t nb = n >= 20 ? 20 : n;
    if (nb >= 2) {
      std::vector<double> vals;
      for (int64_t bI = 0; bI < nb; ++bI) {
        const int64_t lo = bI * n / nb, hi = (bI + 1) * n / nb;
        double sb = 0.0, sd = 0.0;
        for (int64_t i = lo; i < hi; ++i) {
          sb += hist[2 * i];
          sd += hist[2 * i + 1];
        }
        vals.push_back(rho_s2 * (1.0 + sb / sd));
      }
      double mean = 0.0;
      for (double v : vals) mean += v;
      mean /= (double)nb;
      double var = 0.0;
      for (double v : vals) var += (v - mean) * (v - mean);
      var /= (double)(nb - 1);
      *se = std::sqrt(var / (double)nb);
    }
  }
  return ECMC_OK;
}

void to_counters(const RunTotals& t, ecmc_counters_t* out) {
  out->sweeps = t.sweeps;
  out->chains = t.chains;
  out->events = t.events;
  out->lifts = t.lifts;
  out->frozen_hits = t.frozen;
  out->wall_hits = t.walls;
  out->fp64_evals = t.fp64_evals;
  out->sum_b = t.sum_b;
  out->sum_disp = t.sum_disp;
  out->replayed_legs = t.replayed;
  out->rejected_chains = t.rejected;
}

}  // namespace

extern "C" {

const char* ecmc_version(void) { return "ecmc-gb300 0.2 (sm_103a)"; }

const char* ecmc_last_error_message(void) { return g_msg; }

const char* ecmc_strerror(int code) {
  switch (code) {
    case ECMC_OK: return "ok";
    case ECMC_ERR_ARG: return "invalid argument";
    case ECMC_ERR_CUDA: return "CUDA runtime error";
    case ECMC_ERR_OOM: return "out of memory";
    case ECMC_ERR_OVERLAP: return "disks overlap";
    case ECMC_ERR_TIMEOUT: return "device wait timed out";
    case ECMC_ERR_STATE: return "invalid state for this call";
    case ECMC_ERR_CAPACITY: return "cell capacity exceeded";
    case ECMC_ERR_UNSUPPORTED: return "unsupported option";
    case ECMC_ERR_CHAIN_CAP: return "chain event cap reached";
    default: return "unknown error";
  }
}

int ecmc_create(ecmc_t* out, int64_t N, double L, double sigma, int cells_x, int cells_y,
                double ell, uint64_t seed) {
  ecmc_replica_desc_t d;
  d.N = N;
  d.L = L;
  d.sigma = sigma;
  d.cells_x = cells_x;
  d.cells_y = cells_y;
  d.ell = ell;
  d.n_m = 0;
  d.seed = seed;
  d.replica = 0;
  return create_impl(out, &d, 1);
}

int ecmc_create_batch(ecmc_t* out, const ecmc_replica_desc_t* desc, int R) {
  return create_impl(out, desc, R);
}

int ecmc_num_replicas(ecmc_t h, int* R) {
  if (!h || !R) return fail(ECMC_ERR_ARG, "NULL argument");
  *R = h->b.R;
  return ECMC_OK;
}

int ecmc_replica_desc(ecmc_t h, int r, ecmc_replica_desc_t* out) {
  if (!h || !out) return fail(ECMC_ERR_ARG, "NULL argument");
  if (r < 0 || r >= h->b.R) return fail(ECMC_ERR_ARG, "replica out of range");
  const Geom& g = h->geo[r];
  out->N = g.N;
  out->L = g.L;
  out->sigma = g.sigma;
  out->cells_x = g.cells_x;
  out->cells_y = g.cells_y;
  out->ell = g.ell;
  out->n_m = g.n_m;
  out->seed = g.seed;
  out->replica = g.replica;
  return ECMC_OK;
}

int ecmc_destroy(ecmc_t h) {
  if (!h) return ECMC_OK;
  if (h->stream) cudaStreamSynchronize(h->stream);
  free_all(h);
  delete h;
  return ECMC_OK;
}

int ecmc_set_stream(ecmc_t h, void* stream) {
  if (!h) return fail(ECMC_ERR_ARG, "NULL handle");
  CK(cudaStreamSynchronize(h->stream));
  h->stream = stream ? (cudaStream_t)stream : h->own_stream;
  drop_graphs(h);
  return ECMC_OK;
}

int ecmc_set_param(ecmc_t h, int key, double v) {
  if (!h) return fail(ECMC_ERR_ARG, "NULL handle");
  CK(cudaStreamSynchronize(h->stream));
  switch (key) {
    case ECMC_PARAM_N_CHAINS: {
      if (!(v >= 1.0 && v <= 1e6) || v != std::floor(v)) return fail(ECMC_ERR_ARG, "n_m");
      for (Geom& g : h->geo) g.n_m = (int)v;
      drop_graphs(h);
      int rc = upload_geometry(h);
      if (rc) return rc;
      return realloc_chain_recs(h);
    }
    case ECMC_PARAM_DIR_MODE: {
      if (v != 0.0 && v != 1.0 && v != 2.0) return fail(ECMC_ERR_ARG, "direction mode");
      if (v == 2.0 && h->geo[0].boundary == 1)
        return fail(ECMC_ERR_UNSUPPORTED, "the rejecting boundary rule needs axis chains");
      for (Geom& g : h->geo) g.dir_mode = (int)v;
      h->b.iso = v == 2.0 ? 1 : 0;
      drop_graphs(h);
      return compute_layout(h);
    }
    case ECMC_PARAM_PRECISION:
      if (v != 0.0 && v != 1.0) return fail(ECMC_ERR_ARG, "precision");
      h->precision = (int)v;
      for (Geom& g : h->geo) g.precision = (int)v;
      drop_graphs(h);
      return upload_geometry(h);
    case ECMC_PARAM_REPLICA:
      if (!(v >= 0.0) || v != std::floor(v) || v > 9.0e15) return fail(ECMC_ERR_ARG, "replica");
      h->geo[0].replica = (uint64_t)v;
      return upload_geometry(h);
    case ECMC_PARAM_LANES_PER_CELL: {
      const int t = (int)v;
      if ((double)t != v || !(t == 0 || t == 1 || t == 2 || t == 4 || t == 8 || t == 16 || t == 32))
        return fail(ECMC_ERR_ARG, "lanes per cell must be 0 or a power of two <= 32");
      h->tpc_param = t;
      drop_graphs(h);
      return compute_layout(h);
    }
    case ECMC_PARAM_WARPS_PER_BLOCK: {
      const int w = (int)v;
      if ((double)w != v || w < 0 || w > 8) return fail(ECMC_ERR_ARG, "warps per block");
      h->warps_param = w;
      drop_graphs(h);
      return compute_layout(h);
    }
    case ECMC_PARAM_STRIP_WIDTH:
      if (!(v >= 0.125 && v <= 2.0)) return fail(ECMC_ERR_ARG, "strip width");
      h->strip_w = (float)v;
      drop_graphs(h);
      return compute_layout(h);
    case ECMC_PARAM_GR_DR:
      if (!(v > 0.0 && v < 10.0)) return fail(ECMC_ERR_ARG, "g(r) bin width");
      h->gr_dr = v;
      return setup_gr(h);
    case ECMC_PARAM_GR_RMAX:
      if (!(v > h->geo[0].sigma && v < 0.5 * h->geo[0].L)) return fail(ECMC_ERR_ARG, "g(r) range");
      h->gr_rmax = v;
      return setup_gr(h);
    case ECMC_PARAM_TIMING:
      h->timing = v != 0.0;
      return ECMC_OK;
    case ECMC_PARAM_RECORD_CHAINS:
      h->record_chains = v != 0.0;
      drop_graphs(h);
      return realloc_chain_recs(h);
    case ECMC_PARAM_USE_GRAPH:
      h->use_graph = v != 0.0;
      drop_graphs(h);
      return ECMC_OK;
    case ECMC_PARAM_PERSISTENT:
      if (v != 0.0 && v != 1.0) return fail(ECMC_ERR_ARG, "persistent must be 0 or 1");
      h->persist_param = (int)v;
      drop_graphs(h);
      return compute_layout(h);
    case ECMC_PARAM_WAIT_LIMIT_MS:
      if (!(v >= 0.001 && v <= 600000.0)) return fail(ECMC_ERR_ARG, "wait limit out of range");
      h->wait_ms = v;
      h->b.wait_ns = (unsigned long long)(v * 1e6);
      drop_graphs(h);
      return ECMC_OK;
    case ECMC_PARAM_WAIT_TEST:
      if (v != 0.0 && v != 1.0) return fail(ECMC_ERR_ARG, "wait test must be 0 or 1");
      h->b.wait_test = (int)v;
      drop_graphs(h);
      return ECMC_OK;
    case ECMC_PARAM_KERNELS_PER_SWEEP:
      return fail(ECMC_ERR_ARG, "kernels per sweep is read-only");
    case ECMC_PARAM_CHAINS_IN_FLIGHT:
      return fail(ECMC_ERR_ARG, "chains in flight is read-only");
    case ECMC_PARAM_LIST_MODE: {
      if (v != 0.0 && v != 1.0) return fail(ECMC_ERR_ARG, "list mode must be 0 or 1");
      if (v == 1.0)
        for (const Geom& g : h->geo)
          if (g.cap_mem > 128)
            return fail(ECMC_ERR_UNSUPPORTED,
                        "shuffled start lists need cells of at most 128 disks (bound %d)",
                        g.cap_mem);
      for (Geom& g : h->geo) g.list_mode = (int)v;
      drop_graphs(h);
      return upload_geometry(h);
    }
    case ECMC_PARAM_BOUNDARY: {
      if (v != 0.0 && v != 1.0) return fail(ECMC_ERR_ARG, "boundary rule must be 0 or 1");
      if (v == 1.0 && h->b.iso)
        return fail(ECMC_ERR_UNSUPPORTED, "the rejecting boundary rule needs axis chains");
      if (v == 1.0 && !h->undo) {
        const size_t n = (size_t)h->b.C_total * (size_t)h->b.cap;
        if (cudaMalloc(&h->undo, sizeof(UndoEntry) * n) != cudaSuccess) {
          cudaGetLastError();
          h->undo = nullptr;
          return fail(ECMC_ERR_OOM, "undo logs of the rejecting boundary rule (%zu bytes)",
                      sizeof(UndoEntry) * n);
        }
      }
      for (Geom& g : h->geo) {
        g.boundary = (int)v;
        g.undo = h->undo;
        g.undo_stride = h->b.cap;
      }
      h->b.reject = (int)v;
      drop_graphs(h);
      return compute_layout(h);
    }
    case ECMC_PARAM_REPLAY:
      if (v != 0.0 && v != 1.0) return fail(ECMC_ERR_ARG, "replay must be 0 or 1");
      h->b.replay = (int)v;
      drop_graphs(h);
      return ECMC_OK;
    case ECMC_PARAM_FRAME_MODE: {
      const int m = (int)v;
      if ((double)m != v || m < -1 || m > 2) return fail(ECMC_ERR_ARG, "frame mode");
      h->fmode_param = m;
      drop_graphs(h);
      return compute_layout(h);
    }
    default:
      return fail(ECMC_ERR_ARG, "unknown parameter %d", key);
  }
}

int ecmc_get_param(ecmc_t h, int key, double* v) {
  if (!h || !v) return fail(ECMC_ERR_ARG, "NULL argument");
  switch (key) {
    case ECMC_PARAM_N_CHAINS: *v = h->geo[0].n_m; break;
    case ECMC_PARAM_DIR_MODE: *v = h->geo[0].dir_mode; break;
    case ECMC_PARAM_PRECISION: *v = h->precision; break;
    case ECMC_PARAM_REPLICA: *v = (double)h->geo[0].replica; break;
    case ECMC_PARAM_LANES_PER_CELL: *v = h->tpc; break;
    case ECMC_PARAM_GR_DR: *v = h->gr_dr; break;
    case ECMC_PARAM_GR_RMAX: *v = h->gr_rmax; break;
    case ECMC_PARAM_TIMING: *v = h->timing; break;
    case ECMC_PARAM_STRIP_WIDTH: *v = h->strip_w; break;
    case ECMC_PARAM_RECORD_CHAINS: *v = h->record_chains; break;
    case ECMC_PARAM_WARPS_PER_BLOCK: *v = h->warps; break;
    case ECMC_PARAM_USE_GRAPH: *v = h->use_graph; break;
    case ECMC_PARAM_FRAME_MODE: *v = h->fmode; break;
    case ECMC_PARAM_REPLAY: *v = h->b.replay; break;
    case ECMC_PARAM_PERSISTENT: *v = h->persistent; break;
    case ECMC_PARAM_WAIT_LIMIT_MS: *v = h->wait_ms; break;
    case ECMC_PARAM_WAIT_TEST: *v = h->b.wait_test; break;
    case ECMC_PARAM_KERNELS_PER_SWEEP: *v = h->persistent ? 5 : 12; break;
    case ECMC_PARAM_CHAINS_IN_FLIGHT:
      *v = h->persistent ? (double)h->fused_blocks * (32 / h->tpc) : 0.0;
      break;
    case ECMC_PARAM_LIST_MODE: *v = h->geo[0].list_mode; break;
    case ECMC_PARAM_BOUNDARY: *v = h->geo[0].boundary; break;
    default: return fail(ECMC_ERR_ARG, "unknown parameter %d", key);
  }
  return ECMC_OK;
}

int ecmc_set_positions(ecmc_t h, const double* xy, int on_device, int64_t t0) {
  if (!h || !xy) return fail(ECMC_ERR_ARG, "NULL argument");
  if (t0 < 0) return fail(ECMC_ERR_ARG, "t0 < 0");
  CK(cudaStreamSynchronize(h->stream));
  CK(cudaMemcpyAsync(h->xy_tmp, xy, sizeof(double) * 2 * (size_t)h->b.N_total,
                     on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream));
  return load_positions_dev(h, h->xy_tmp, t0);
}

int ecmc_sweep(ecmc_t h, int64_t n) {
  if (!h) return fail(ECMC_ERR_ARG, "NULL handle");
  if (n < 0) return fail(ECMC_ERR_ARG, "n < 0");
  if (!h->valid_state) return fail(ECMC_ERR_STATE, "state invalid after an earlier error");
  int rc = ensure_history(h, n);
  if (rc) return rc;
  const bool graph = h->use_graph && !h->timing;
  for (int64_t i = 0; i < n; ++i) {
    if (graph) {
      const int par = h->b.cur;
      if (!h->graph[par]) {
        cudaGraph_t gr;
        CK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
        const int cur0 = h->b.cur;
        rc = enqueue_sweep(h);
        h->b.cur = cur0;
        cudaError_t e = cudaStreamEndCapture(h->stream, &gr);
        if (rc) return rc;
        if (e != cudaSuccess)
          return fail(ECMC_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(e));
        e = cudaGraphInstantiate(&h->graph[par], gr, 0);
        cudaGraphDestroy(gr);
        if (e != cudaSuccess)
          return fail(ECMC_ERR_CUDA, "graph instantiation failed: %s", cudaGetErrorString(e));
        for (int c = 0; c < 4; ++c) h->launches[c] -= (c == TC_FRAME || c == TC_PHASE) ? 4 : 1;
      }
      CK(cudaGraphLaunch(h->graph[par], h->stream));
      h->launches[TC_BIN] += 1;
      h->launches[TC_FRAME] += 4;
      h->launches[TC_PHASE] += 4;
      h->launches[TC_OTHER] += 1;
      h->b.cur = 1 - par;
    } else {
      rc = enqueue_sweep(h);
      if (rc) return rc;
    }
    h->t_host += 1;
    h->hist_len_host += 1;
  }
  return ECMC_OK;
}

int ecmc_synchronize(ecmc_t h) {
  if (!h) return fail(ECMC_ERR_ARG, "NULL handle");
  return check_device_error(h);
}

int ecmc_positions(ecmc_t h, double* xy_out, int on_device) {
  if (!h || !xy_out) return fail(ECMC_ERR_ARG, "NULL argument");
  const size_t bytes = sizeof(double) * 2 * (size_t)h->b.N_total;
  if (on_device) {
    launch_gather(h->b, xy_out, h->stream);
  } else {
    launch_gather(h->b, h->xy_tmp, h->stream);
    CK(cudaMemcpyAsync(xy_out, h->xy_tmp, bytes, cudaMemcpyDeviceToHost, h->stream));
  }
  CK(cudaGetLastError());
  return check_device_error(h);
}

int ecmc_sweep_index(ecmc_t h, int64_t* t) {
  if (!h || !t) return fail(ECMC_ERR_ARG, "NULL argument");
  *t = h->t_host;
  return ECMC_OK;
}

int ecmc_counters(ecmc_t h, ecmc_counters_t* out) {
  if (!h || !out) return fail(ECMC_ERR_ARG, "NULL argument");
  std::vector<RunTotals> t(h->b.R);
  CK(cudaMemcpyAsync(t.data(), h->b.totals, sizeof(RunTotals) * t.size(), cudaMemcpyDeviceToHost,
                     h->stream));
  int rc = check_device_error(h);
  if (rc) return rc;
  RunTotals s;
  std::memset(&s, 0, sizeof(s));
  for (const RunTotals& v : t) {
    s.sum_b += v.sum_b;
    s.sum_disp += v.sum_disp;
    s.sweeps = v.sweeps;
    s.chains += v.chains;
    s.events += v.events;
    s.lifts += v.lifts;
    s.frozen += v.frozen;
    s.walls += v.walls;
    s.fp64_evals += v.fp64_evals;
    s.replayed += v.replayed;
    s.rejected += v.rejected;
  }
  to_counters(s, out);
  return ECMC_OK;
}

int ecmc_replica_counters(ecmc_t h, int r, ecmc_counters_t* out) {
  if (!h || !out) return fail(ECMC_ERR_ARG, "NULL argument");
  if (r < 0 || r >= h->b.R) return fail(ECMC_ERR_ARG, "replica out of range");
  RunTotals t;
  CK(cudaMemcpyAsync(&t, h->b.totals + r, sizeof(t), cudaMemcpyDeviceToHost, h->stream));
  int rc = check_device_error(h);
  if (rc) return rc;
  to_counters(t, out);
  return ECMC_OK;
}

int ecmc_reset_stats(ecmc_t h) {
  if (!h) return fail(ECMC_ERR_ARG, "NULL handle");
  CK(cudaStreamSynchronize(h->stream));
  CK(cudaMemsetAsync(h->b.totals, 0, sizeof(RunTotals) * h->b.R, h->stream));
  const int64_t zero = 0;
  for (int r = 0; r < h->b.R; ++r)
    CK(cudaMemcpyAsync((char*)(h->b.state + r) + offsetof(SweepState, history_len), &zero,
                       sizeof(zero), cudaMemcpyHostToDevice, h->stream));
  h->hist_len_host = 0;
  CK(cudaMemsetAsync(h->gr_counts, 0, sizeof(unsigned long long) * h->gr_nbins * h->geo.size(),
                     h->stream));
  h->gr_meas.assign(h->geo.size(), 0);
  CK(cudaStreamSynchronize(h->stream));
  if (h->timing) harvest_timing(h);
  for (int c = 0; c < 4; ++c) {
    h->ms[c] = 0.0;
    h->launches[c] = 0;
  }
  return ECMC_OK;
}

int ecmc_pressure(ecmc_t h, double* betaP, double* se) {
  if (!h || !betaP) return fail(ECMC_ERR_ARG, "NULL argument");
  return pressure_of(h, 0, betaP, se);
}

int ecmc_replica_pressure(ecmc_t h, int r, double* betaP, double* se) {
  if (!h || !betaP) return fail(ECMC_ERR_ARG, "NULL argument");
  if (r < 0 || r >= h->b.R) return fail(ECMC_ERR_ARG, "replica out of range");
  return pressure_of(h, r, betaP, se);
}

int ecmc_gr_measure(ecmc_t h) { return ecmc_replica_gr_measure(h, 0); }

int ecmc_replica_gr_measure(ecmc_t h, int r) {
  if (!h) return fail(ECMC_ERR_ARG, "NULL handle");
  const int R = (int)h->geo.size();
  if (r < -1 || r >= R) return fail(ECMC_ERR_ARG, "replica %d out of range", r);
  const int r0 = r < 0 ? 0 : r, r1 = r < 0 ? R : r + 1;
  for (int q = r0; q < r1; ++q) {
    launch_gr(h->geo[q], h->b, h->gr_dr, h->gr_nbins, h->gr_counts + (size_t)q * h->gr_nbins,
              h->stream);
    h->gr_meas[q] += 1;
  }
  CK(cudaGetLastError());
  return ECMC_OK;
}

int ecmc_hexatic(ecmc_t h, double rs, double* psi, double* psi_k, int32_t* n_nb,
                 int64_t* n_bad) {
  if (!h || !psi) return fail(ECMC_ERR_ARG, "NULL argument");
  if (!h->valid_state) return fail(ECMC_ERR_STATE, "state invalid after an earlier error");
  for (const Geom& g : h->geo) {
    const double r = rs > 0.0 ? rs : 3.5 * g.sigma;
    if (!(g.L > 2.0 * r)) return fail(ECMC_ERR_ARG, "box side must exceed 2 rs");
  }
  const int64_t N = h->b.N_total;
  unsigned long long* bad = h->u64_tmp + 1;
  CK(cudaMemsetAsync(bad, 0, sizeof(unsigned long long), h->stream));
  double2* pk = reinterpret_cast<double2*>(h->xy_tmp);
  if (launch_hexatic(h->b, rs, pk, h->int_tmp, bad, h->stream))
    return fail(ECMC_ERR_CUDA, "hexatic kernel launch failed: %s",
                cudaGetErrorString(cudaGetLastError()));
  std::vector<double> hk(2 * (size_t)N);
  std::vector<int32_t> hn((size_t)N);
  unsigned long long hb = 0;
  CK(cudaMemcpyAsync(hk.data(), pk, sizeof(double) * 2 * (size_t)N, cudaMemcpyDeviceToHost,
                     h->stream));
  CK(cudaMemcpyAsync(hn.data(), h->int_tmp, sizeof(int32_t) * (size_t)N, cudaMemcpyDeviceToHost,
                     h->stream));
  CK(cudaMemcpyAsync(&hb, bad, sizeof(hb), cudaMemcpyDeviceToHost, h->stream));
  int rc = check_device_error(h);
  if (rc) return rc;
  for (size_t r = 0; r < h->geo.size(); ++r) {
    const int64_t a = h->n_off[r], e = h->n_off[r + 1];
    double sre = 0.0, sim = 0.0;
    for (int64_t k = a; k < e; ++k) {
      if (hn[k] < 0)
        return fail(ECMC_ERR_CAPACITY, "more than 64 disks within rs of disk %lld of replica %d",
                    (long long)(k - a), (int)r);
      sre += hk[2 * k];
      sim += hk[2 * k + 1];
    }
    psi[2 * r] = sre / (double)(e - a);
    psi[2 * r + 1] = sim / (double)(e - a);
  }
  if (psi_k) std::memcpy(psi_k, hk.data(), sizeof(double) * 2 * (size_t)N);
  if (n_nb) std::memcpy(n_nb, hn.data(), sizeof(int32_t) * (size_t)N);
  if (n_bad) *n_bad = (int64_t)hb;
  return ECMC_OK;
}

int ecmc_gr_nbins(ecmc_t h, int* nbins) {
  if (!h || !nbins) return fail(ECMC_ERR_ARG, "NULL argument");
  *nbins = h->gr_nbins;
  return ECMC_OK;
}

int ecmc_gr_counts(ecmc_t h, int64_t* counts, int nbins, int64_t* n_meas) {
  return ecmc_replica_gr_counts(h, 0, counts, nbins, n_meas);
}

int ecmc_replica_gr_counts(ecmc_t h, int r, int64_t* counts, int nbins, int64_t* n_meas) {
  if (!h || !counts) return fail(ECMC_ERR_ARG, "NULL argument");
  if (r < 0 || r >= (int)h->geo.size()) return fail(ECMC_ERR_ARG, "replica %d out of range", r);
  if (nbins != h->gr_nbins) return fail(ECMC_ERR_ARG, "nbins must be %d", h->gr_nbins);
  CK(cudaMemcpyAsync(counts, h->gr_counts + (size_t)r * h->gr_nbins, sizeof(int64_t) * nbins,
                     cudaMemcpyDeviceToHost, h->stream));
  int rc = check_device_error(h);
  if (rc) return rc;
  if (n_meas) *n_meas = h->gr_meas[r];
  return ECMC_OK;
}

int ecmc_gr(ecmc_t h, double* g_out, double* r_out, int nbins) {
  return ecmc_replica_gr(h, 0, g_out, r_out, nbins);
}

int ecmc_replica_gr(ecmc_t h, int r, double* g_out, double* r_out, int nbins) {
  if (!h || !g_out) return fail(ECMC_ERR_ARG, "NULL argument");
  std::vector<int64_t> c(nbins > 0 ? nbins : 1);
  int64_t nm = 0;
  int rc = ecmc_replica_gr_counts(h, r, c.data(), nbins, &nm);
  if (rc) return rc;
  if (nm < 1) return fail(ECMC_ERR_STATE, "no g(r) measurement yet");
  const Geom& g = h->geo[r];
  const double pi = 3.14159265358979323846;
  const double N = (double)g.N, rho = N / (g.L * g.L), dr = h->gr_dr;
  for (int i = 0; i < nbins; ++i) {
    const double e0 = g.sigma + dr * i, e1 = e0 + dr;
    const double R = 2.0 * (e1 * e1 * e1 - e0 * e0 * e0) / (3.0 * (e1 * e1 - e0 * e0));
    g_out[i] = ((double)c[i] / (double)nm) / (N * rho * 2.0 * pi * R * dr);
    if (r_out) r_out[i] = R;
  }
  return ECMC_OK;
}

int ecmc_min_distance(ecmc_t h, double* dmin) {
  if (!h || !dmin) return fail(ECMC_ERR_ARG, "NULL argument");
  double d2 = 0.0;
  int rc = min_dist2(h, &d2);
  if (rc) return rc;
  *dmin = std::sqrt(d2);
  return ECMC_OK;
}

int ecmc_last_cells(ecmc_t h, int32_t* cell_of_id) {
  if (!h || !cell_of_id) return fail(ECMC_ERR_ARG, "NULL argument");
  for (const Geom& g : h->geo) launch_cells_of(g, h->b, h->int_tmp + g.n_off, h->stream);
  CK(cudaMemcpyAsync(cell_of_id, h->int_tmp, sizeof(int) * (size_t)h->b.N_total,
                     cudaMemcpyDeviceToHost, h->stream));
  return check_device_error(h);
}

int ecmc_kernel_times(ecmc_t h, ecmc_timing_t* out) {
  if (!h || !out) return fail(ECMC_ERR_ARG, "NULL argument");
  CK(cudaStreamSynchronize(h->stream));
  harvest_timing(h);
  out->bin_ms = h->ms[TC_BIN];
  out->frame_ms = h->ms[TC_FRAME];
  out->phase_ms = h->ms[TC_PHASE];
  out->other_ms = h->ms[TC_OTHER];
  out->bin_launches = h->launches[TC_BIN];
  out->frame_launches = h->launches[TC_FRAME];
  out->phase_launches = h->launches[TC_PHASE];
  out->other_launches = h->launches[TC_OTHER];
  return ECMC_OK;
}

int ecmc_chain_records(ecmc_t h, ecmc_chain_rec_t* out, int64_t n) {
  if (!h || !out) return fail(ECMC_ERR_ARG, "NULL argument");
  if (!h->record_chains || !h->b.chain_recs) return fail(ECMC_ERR_STATE, "records are off");
  const Geom& g = h->geo[0];
  if (n != (int64_t)g.ncell * g.n_m) return fail(ECMC_ERR_ARG, "n must be cells * n_m");
  static_assert(sizeof(ChainRec) == sizeof(ecmc_chain_rec_t), "record layout");
  CK(cudaMemcpy2DAsync(out, sizeof(ChainRec) * g.n_m, h->b.chain_recs,
                       sizeof(ChainRec) * h->b.rec_stride, sizeof(ChainRec) * g.n_m, g.ncell,
                       cudaMemcpyDeviceToHost, h->stream));
  return check_device_error(h);
}

int ecmc_suggest_parameters(int64_t N, double L, double sigma, double min_cell_side,
                            ecmc_replica_desc_t* out) {
  if (!out || N < 1 || !(L > 0.0) || !(sigma > 0.0)) return fail(ECMC_ERR_ARG, "bad arguments");
  const double pi = 3.14159265358979323846;
  const double eta = (double)N * pi * sigma * sigma / (4.0 * L * L);  // eq. (1)
  const double eta_hcp = pi / (2.0 * std::sqrt(3.0));
  const double lambda0 = sigma * (eta_hcp - eta) / (2.0 * eta_hcp);   // Sec. 4
  if (!(lambda0 > 0.0)) return fail(ECMC_ERR_ARG, "packing fraction above close packing");
  const double side_min = min_cell_side > sigma ? min_cell_side : sigma;
  // step 1: largest n with N / (eta n) > 100
  double n_max = (double)N / (100.0 * eta);
  long long half = (long long)std::floor(std::sqrt(n_max > 1.0 ? n_max : 1.0));
  if ((double)half * (double)half * 100.0 * eta >= (double)N && half > 1) --half;
  if (half < 1) half = 1;
  int cells = (int)(2 * half);
  while (cells > 2 && !(L / cells > side_min)) cells -= 2;
  if (!(L / cells > side_min)) return fail(ECMC_ERR_ARG, "box too small for 2x2 cells");
  const double n = (double)cells * (double)cells / 4.0;
  // step 2: eq. (criterion), ell = lambda0 (N / (eta n))^(1/2)
  const double ell = lambda0 * std::sqrt((double)N / (eta * n));
  // step 3: eq. (nm)
  const double nm = (double)N / (4.0 * n) * lambda0 / ell;
  const double nmr = std::floor(nm + 0.5);
  out->N = N;
  out->L = L;
  out->sigma = sigma;
  out->cells_x = cells;
  out->cells_y = cells;
  out->ell = ell;
  out->n_m = nmr < 1.0 ? 1 : (int)nmr;
  return ECMC_OK;
}

int ecmc_autotune(ecmc_t h, int trial_sweeps, ecmc_tune_result_t* best, ecmc_tune_result_t* all,
                  int max_all, int* n_all) {
  if (!h || !best || trial_sweeps < 1) return fail(ECMC_ERR_ARG, "bad arguments");
  if (!h->valid_state) return fail(ECMC_ERR_STATE, "state invalid after an earlier error");
  CK(cudaStreamSynchronize(h->stream));
  // save the state
  const size_t pos_bytes = sizeof(double) * 2 * (size_t)h->b.N_total;
  double* saved = nullptr;
  RunTotals* saved_tot = nullptr;
  CK(cudaMalloc(&saved, pos_bytes));
  if (cudaMalloc(&saved_tot, sizeof(RunTotals) * h->b.R) != cudaSuccess) {
    cudaFree(saved);
    return fail(ECMC_ERR_OOM, "autotune scratch");
  }
  launch_gather(h->b, saved, h->stream);
  cudaMemcpyAsync(saved_tot, h->b.totals, sizeof(RunTotals) * h->b.R, cudaMemcpyDeviceToDevice,
                  h->stream);
  const int64_t t_saved = h->t_host, hist_saved = h->hist_len_host;
  const int tpc0 = h->tpc_param, warps0 = h->warps_param, timing0 = h->timing;
  const int fmode0 = h->fmode_param, persist0 = h->persist_param;
  h->timing = 0;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  std::vector<ecmc_tune_result_t> res;
  int rc = ECMC_OK;
  const int tpcs[6] = {1, 2, 4, 8, 16, 32};
  const int wps[2] = {1, 2};
  // the persistent sweep kernel for every lanes-per-cell choice and both
  // placements of the FP64 coordinates (warps per block do not apply to it),
  // then the per-phase kernels for every shape
  for (int pm = 1; pm >= 0 && rc == ECMC_OK; --pm)
  for (int fm = 0; fm < 3 && rc == ECMC_OK; ++fm)
  for (int ti = 0; ti < 6 && rc == ECMC_OK; ++ti)
    for (int wi = 0; wi < 2 && rc == ECMC_OK; ++wi) {
      if (pm == 1 && (fm > 1 || wi > 0)) continue;
      h->persist_param = pm;
      h->tpc_param = tpcs[ti];
      h->warps_param = wps[wi];
      h->fmode_param = fm;
      drop_graphs(h);
      if (compute_layout(h) != ECMC_OK) {
        cudaGetLastError();
        continue;
      }
      if (h->persistent != pm || h->fmode != fm) continue;
      if (!pm && h->warps != wps[wi]) continue;
      if (!pm && fm == 2 && res.size() > 0) continue;  // global frames only when nothing else fits
      rc = ecmc_sweep(h, 1);
      if (rc) break;
      cudaEventRecord(e0, h->stream);
      rc = ecmc_sweep(h, trial_sweeps);
      if (rc) break;
      cudaEventRecord(e1, h->stream);
      rc = check_device_error(h);
      if (rc) break;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      ecmc_tune_result_t r;
      r.lanes_per_cell = h->tpc;
      r.warps_per_block = h->warps;
      r.frame_mode = h->fmode;
      r.persistent = h->persistent;
      r.ms_per_sweep = ms / trial_sweeps;
      res.push_back(r);
      // back to the saved state before the next shape
      h->hist_len_host = hist_saved;
      rc = load_positions_dev(h, saved, t_saved);
      cudaMemcpyAsync(h->b.totals, saved_tot, sizeof(RunTotals) * h->b.R,
                      cudaMemcpyDeviceToDevice, h->stream);
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  h->timing = timing0;
  int bi = -1;
  for (size_t i = 0; i < res.size(); ++i)
    if (bi < 0 || res[i].ms_per_sweep < res[bi].ms_per_sweep) bi = (int)i;
  if (rc == ECMC_OK && bi < 0) rc = fail(ECMC_ERR_UNSUPPORTED, "no launch shape fits");
  if (rc == ECMC_OK) {
    *best = res[bi];
    h->tpc_param = res[bi].lanes_per_cell;
    h->warps_param = res[bi].warps_per_block;
    h->fmode_param = res[bi].frame_mode;
    h->persist_param = res[bi].persistent;
  } else {
    h->tpc_param = tpc0;
    h->warps_param = warps0;
    h->fmode_param = fmode0;
    h->persist_param = persist0;
  }
  drop_graphs(h);
  int rc2 = compute_layout(h);
  h->hist_len_host = hist_saved;
  int rc3 = load_positions_dev(h, saved, t_saved);
  cudaMemcpyAsync(h->b.totals, saved_tot, sizeof(RunTotals) * h->b.R, cudaMemcpyDeviceToDevice,
                  h->stream);
  cudaStreamSynchronize(h->stream);
  cudaFree(saved);
  cudaFree(saved_tot);
  if (all && n_all) {
    const int n = (int)res.size() < max_all ? (int)res.size() : max_all;
    for (int i = 0; i < n; ++i) all[i] = res[i];
    *n_all = n;
  } else if (n_all) {
    *n_all = (int)res.size();
  }
  if (rc) return rc;
  if (rc2) return rc2;
  return rc3;
}

int ecmc_device_peaks(double* smem_gbs, double* fp64_gflops) {
  if (!smem_gbs || !fp64_gflops) return fail(ECMC_ERR_ARG, "NULL argument");
  if (probe_peaks(smem_gbs, fp64_gflops))
    return fail(ECMC_ERR_CUDA, "peak probe failed: %s", cudaGetErrorString(cudaGetLastError()));
  return ECMC_OK;
}

int ecmc_sqrt_rn(const double* x, double* out, int64_t n, int where, double rel_error,
                 void* stream) {
  if (n < 0 || (n > 0 && (!x || !out))) return fail(ECMC_ERR_ARG, "bad arguments");
  if (where == 0) {
    if (!(std::fabs(rel_error) <= std::ldexp(1.0, -20)))
      return fail(ECMC_ERR_ARG, "rel_error must be within 2^-20");
    host_sqrt_rn(x, out, n, rel_error);
    return ECMC_OK;
  }
  if (where != 1) return fail(ECMC_ERR_ARG, "where must be 0 (host) or 1 (device)");
  cudaStream_t s = (cudaStream_t)stream;
  if (launch_sqrt_rn(x, out, n, s) || cudaStreamSynchronize(s) != cudaSuccess)
    return fail(ECMC_ERR_CUDA, "square-root kernel failed: %s",
                cudaGetErrorString(cudaGetLastError()));
  return ECMC_OK;
}

}  // extern "C"
