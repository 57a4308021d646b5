// ecmc_noalloc.cu -- ecmc_sweep_noalloc: sweeps of a caller-held system
// without any device allocation.
//
// Some callers cannot allocate device memory: an application whose device
// memory is owned by its own pool (every cudaMalloc outside it is forbidden),
// or code that must not allocate once its set-up phase is over.  This entry
// point runs the same kernels as ecmc_sweep, but all of its scratch memory
// (cell buckets, frame records, per-cell results, sweep state) is carved out
// of one file-scope __device__ array of ECMC_NOALLOC_SCRATCH_BYTES bytes that
// is part of the library image: every GPU that loads the library holds it
// until the process exits.  The caller passes the positions (device memory,
// read and overwritten) and the system's parameters.
//
// The array is shared by every call: calls that overlap on the GPU (on
// different streams, or from different host threads) race on it and must be
// serialised by the caller.  What must start at zero (bucket counts,
// running totals, the error word) is cleared by every call; the rest is
// written before it is read.
#include <cmath>
#include <cstring>
#include <mutex>

#include "ecmc.h"
#include "ecmc_internal.cuh"

using namespace ecmc;

static __device__ __align__(256) unsigned char g_noalloc_scratch[ECMC_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
unsigned char* g_noalloc_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device.  In host code
// the name g_noalloc_scratch is only a host-side stand-in, so the address is
// looked up once per device (with that device current) and cached.
int scratch_address(unsigned char** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return ECMC_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr)
      return ECMC_ERR_CUDA;
    g_noalloc_ptr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_noalloc_ptr[dev];
  return ECMC_OK;
}

size_t carve(size_t& off, size_t bytes) {
  const size_t at = (off + 255) & ~size_t(255);
  off = at + bytes;
  return at;
}

double packing(double W, double H, double sigma) {
  const double sp = sigma * (1.0 - 1e-6);
  return (W + sp) * (H + sp) / (3.14159265358979323846 * sp * sp / 4.0);
}

}  // namespace

extern "C" int ecmc_sweep_noalloc(double* xy, int64_t N, double L, double sigma, int cells_x,
                                  int cells_y, double ell, int n_m, uint64_t seed,
                                  uint64_t replica, int64_t t0, int64_t n_sweeps, void* stream) {
  if (!xy || N < 1 || N >= (int64_t(1) << 27) || !(L > 0.0) || !(sigma > 0.0) ||
      !std::isfinite(L) || cells_x < 2 || cells_y < 2 || (cells_x & 1) || (cells_y & 1) ||
      !(L / cells_x > sigma) || !(L / cells_y > sigma) || !(ell >= 0.0) || !std::isfinite(ell) ||
      n_m < 1 || t0 < 0 || n_sweeps < 0 || !(sigma >= std::ldexp(1.0, -40)) ||
      !(sigma <= std::ldexp(1.0, 40)) || !(L < std::ldexp(sigma, 40)))
    return ECMC_ERR_ARG;

  // geometry and capacities, as for a handle
  Geom g;
  std::memset(&g, 0, sizeof(g));
  g.N = N;
  g.L = L;
  g.sigma = sigma;
  g.sig2 = sigma * sigma;
  g.cells_x = cells_x;
  g.cells_y = cells_y;
  g.ncell = cells_x * cells_y;
  g.w = L / (double)cells_x;
  g.h = L / (double)cells_y;
  g.inv_w = 1.0 / g.w;
  g.inv_h = 1.0 / g.h;
  set_bin_screen(g);
  g.ell = ell;
  g.n_m = n_m;
  g.seed = seed;
  g.replica = replica;
  g.dir_mode = 0;
  g.precision = 1;
  g.nact = (cells_x / 2) * (cells_y / 2);
  g.cap_mem = (int)std::floor(packing(g.w, g.h, sigma)) + 2;
  g.cap_obj = (int)std::floor(packing(g.w + 2 * sigma, g.h + 2 * sigma, sigma)) + 2;
  if (g.cap_mem > g.cap_obj) g.cap_mem = g.cap_obj;
  if ((int64_t)g.ncell * g.cap_mem < N) return ECMC_ERR_ARG;
  {
    const double ext = (g.w > g.h ? g.w : g.h) + 1.01 * sigma;
    double M = 1.0;
    while (M < ext) M *= 2.0;
    const double e = 6.5 * std::ldexp(1.0, -24) * M;
    const double ex = (2.0 * sigma + 2.0 * e) * e + 3.0 * std::ldexp(1.0, -24) * sigma * sigma;
    g.eps_d = (float)(e * 1.0000001);
    g.s_margin = (float)(1.25 * (e + std::sqrt(ex) + std::ldexp(1.0, -20) * sigma +
                                 std::ldexp(1.0, -23) * (2.0 * M + sigma)));
    g.sig_plus = std::nextafter((float)(sigma + e + std::ldexp(sigma, -40)), 1e30f);
    g.sig_minus = std::nextafter((float)(sigma - e - std::ldexp(sigma, -40)), -1e30f);
    g.sig2f = (float)(sigma * sigma);
    g.sigf = (float)sigma;
    g.strip_margin = (float)(4.0 * e + 1e-5 * sigma);
    const double bw = 0.5 * sigma;
    g.nbin = (int)std::ceil(((g.w > g.h ? g.w : g.h) + 2.0 * sigma) / bw) + 1;
    g.bin_w = (float)bw;
    g.inv_bin_w = (float)(1.0 / bw);
  }
  int tpc = 32;
  for (int t = 4; t <= 32; t *= 2) {
    if (phase_smem_bytes(make_layout(32 / t, g.nbin, g.cap_mem, g.cap_obj), 1, 0) <= 52 * 1024) {
      tpc = t;
      break;
    }
  }
  const RecLayout lay = make_layout(32 / tpc, g.nbin, g.cap_mem, g.cap_obj);
  if (phase_smem_bytes(lay, 1, 0) > 232448 || frame_build_smem(lay) > 232448)
    return ECMC_ERR_UNSUPPORTED;

  // carve the scratch array
  const size_t slots = (size_t)g.ncell * g.cap_mem;
  const int n_active = (cells_x / 2) * (cells_y / 2);
  const int n_groups = (n_active + lay.cpw - 1) / lay.cpw;
  size_t off = 0;
  size_t o_px[2], o_py[2], o_pid[2], o_cnt[2];
  for (int i = 0; i < 2; ++i) {
    o_px[i] = carve(off, sizeof(double) * slots);
    o_py[i] = carve(off, sizeof(double) * slots);
    o_pid[i] = carve(off, sizeof(int) * slots);
    o_cnt[i] = carve(off, sizeof(int) * (size_t)g.ncell);
  }
  const size_t o_state = carve(off, sizeof(SweepState));
  const size_t o_stats = carve(off, sizeof(CellStats) * (size_t)g.ncell);
  const size_t o_tot = carve(off, sizeof(RunTotals));
  const size_t o_err = carve(off, sizeof(int));
  const size_t o_rec = carve(off, (size_t)n_groups * lay.bytes);
  const size_t o_geo = carve(off, sizeof(Geom));
  const size_t o_crep = carve(off, sizeof(int) * (size_t)g.ncell);
  const size_t o_arep = carve(off, sizeof(int) * (size_t)n_active);
  const size_t o_noff = carve(off, sizeof(int64_t) * 2);
  const int n_chunks = (g.ncell + 2047) / 2048;
  const size_t o_chunks = carve(off, sizeof(int2) * (size_t)n_chunks);
  const size_t o_choff = carve(off, sizeof(int) * 2);
  const size_t o_part = carve(off, sizeof(ChunkSums) * (size_t)n_chunks);
  // larger systems than the static array can serve are rejected up front
  if (off > (size_t)ECMC_NOALLOC_SCRATCH_BYTES) return ECMC_ERR_CAPACITY;

  unsigned char* base = nullptr;
  if (scratch_address(&base) != ECMC_OK) return ECMC_ERR_CUDA;
  DevBufs b;
  std::memset(&b, 0, sizeof(b));
  b.replay = 1;
  for (int i = 0; i < 2; ++i) {
    b.px[i] = reinterpret_cast<double*>(base + o_px[i]);
    b.py[i] = reinterpret_cast<double*>(base + o_py[i]);
    b.pid[i] = reinterpret_cast<int*>(base + o_pid[i]);
    b.count[i] = reinterpret_cast<int*>(base + o_cnt[i]);
  }
  b.state = reinterpret_cast<SweepState*>(base + o_state);
  b.cell_stats = reinterpret_cast<CellStats*>(base + o_stats);
  b.totals = reinterpret_cast<RunTotals*>(base + o_tot);
  b.err = reinterpret_cast<int*>(base + o_err);
  b.records = base + o_rec;
  b.history = nullptr;
  b.history_cap = 0;
  b.chain_recs = nullptr;
  b.rec_stride = n_m;
  b.cur = 0;
  b.rg = reinterpret_cast<Geom*>(base + o_geo);
  b.cell_rep = reinterpret_cast<int*>(base + o_crep);
  b.act_rep = reinterpret_cast<int*>(base + o_arep);
  b.n_off = reinterpret_cast<int64_t*>(base + o_noff);
  b.R = 1;
  b.C_total = g.ncell;
  b.A_total = n_active;
  b.cap = g.cap_mem;
  b.N_total = N;
  b.chunks = reinterpret_cast<int2*>(base + o_chunks);
  b.chunk_off = reinterpret_cast<int*>(base + o_choff);
  b.partials = reinterpret_cast<ChunkSums*>(base + o_part);
  b.n_chunks = n_chunks;
  b.fmode = 0;
  const int64_t n_off_host[2] = {0, N};
  const int chunk_off_host[2] = {0, n_chunks};

  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (configure_frame_build(lay) || configure_phase(lay, tpc, 1, 0)) return ECMC_ERR_CUDA;

  // clear what must start at zero, set the sweep counter
  SweepState st;
  std::memset(&st, 0, sizeof(st));
  st.t = t0;
  if (cudaMemsetAsync(b.count[0], 0, sizeof(int) * (size_t)g.ncell, s) != cudaSuccess ||
      cudaMemsetAsync(b.count[1], 0, sizeof(int) * (size_t)g.ncell, s) != cudaSuccess ||
      cudaMemsetAsync(b.totals, 0, sizeof(RunTotals), s) != cudaSuccess ||
      cudaMemsetAsync(b.err, 0, sizeof(int), s) != cudaSuccess ||
      cudaMemsetAsync((void*)b.cell_rep, 0, sizeof(int) * (size_t)g.ncell, s) != cudaSuccess ||
      cudaMemsetAsync((void*)b.act_rep, 0, sizeof(int) * (size_t)n_active, s) != cudaSuccess ||
      cudaMemcpyAsync((void*)b.rg, &g, sizeof(g), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync((void*)b.n_off, n_off_host, sizeof(n_off_host), cudaMemcpyHostToDevice,
                      s) != cudaSuccess ||
      cudaMemcpyAsync(b.state, &st, sizeof(st), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync((void*)b.chunk_off, chunk_off_host, sizeof(chunk_off_host),
                      cudaMemcpyHostToDevice, s) != cudaSuccess)
    return ECMC_ERR_CUDA;
  for (int k = 0; k < n_chunks; ++k) {
    const int2 ch = make_int2(k * 2048, (k + 1) * 2048 < g.ncell ? (k + 1) * 2048 : g.ncell);
    if (cudaMemcpyAsync((void*)(b.chunks + k), &ch, sizeof(ch), cudaMemcpyHostToDevice, s) !=
        cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
      return ECMC_ERR_CUDA;
  }
  if (cudaStreamSynchronize(s) != cudaSuccess) return ECMC_ERR_CUDA;

  // caller positions -> buckets, n sweeps, buckets -> caller positions
  launch_load_flat(b, xy, s);
  launch_sweep_begin(b, s);
  launch_bin(b, -1, b.cur, s);
  for (int64_t i = 0; i < n_sweeps; ++i) {
    const int src = b.cur, dst = 1 - b.cur;
    launch_sweep_begin(b, s);
    launch_bin(b, src, dst, s);
    b.cur = dst;
    for (int ci = 0; ci < 4; ++ci) {
      launch_frame_build(b, lay, ci, s);
      if (launch_phase(b, lay, ci, tpc, 1, 0, 1, s)) return ECMC_ERR_CUDA;
    }
    launch_sweep_end(b, s);
  }
  launch_gather(b, xy, s);
  if (cudaGetLastError() != cudaSuccess) return ECMC_ERR_CUDA;
  int err = 0;
  if (cudaMemcpyAsync(&err, b.err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return ECMC_ERR_CUDA;
  if (err == DEV_CAPACITY) return ECMC_ERR_CAPACITY;
  if (err == DEV_CHAIN_CAP) return ECMC_ERR_CHAIN_CAP;
  return ECMC_OK;
}
